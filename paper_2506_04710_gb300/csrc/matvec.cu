// The FFT product with the two-level block-Toeplitz part A and the edge
// coupling (B, B^T, C) of Z = [[A, B^T], [B, C]] (Sec. II-C, Eq. matrixForm,
// Eq. submatrixAA).
//
// Pipeline for y = Z' x (x, y: [nrhs][N], Toeplitz part [ny][nx][b] per RHS):
//   1. x pass  : X1[r][n][kx][i]  = FFT_m( x[r][n][m][i], zero-padded to lx )
//   2. y pass  : Xh[f][r][i]      = FFT_n( X1[r][n][kx][i], zero-padded to ly ), f = ky*lx+kx
//   3. product : Xh[f] <- T^[f] Xh[f],  Xh[-f] <- T^[f]^T Xh[-f]   (in place, one T^ read per pair)
//   4. y pass^-1: X1[r][n][kx][i] = IFFT_ky(Xh)[n],  n < ny (crop)
//   5. x pass^-1: y[r][n][m][i]   = IFFT_kx(X1)[m] / (lx ly) + (B^T x_E)[...],  m < nx (crop),
//                 absent elements pass x through (identity rows)
//   side branch (concurrent with 1-4): B x_T and B^T x_E in one pass over B,
//                 then y_E = sum of partials + C x_E.
#include <algorithm>

#include "common.cuh"
#include "fft.cuh"
#include "fftreg.cuh"
#include "passes.cuh"
#include "tma.cuh"
#include "tcgemm.cuh"

namespace ztoep {

// ------------------------------------------------------------ block product
// One CTA per frequency pair {f, -f}: T^[f] (b x b, row-major) is staged in
// shared memory once and used for both Yh[f] <- T^[f] Xh[f] (row products,
// each thread walks its row with a skew so that a warp hits distinct banks)
// and Yh[-f] <- T^[f]^T Xh[-f] (column products, contiguous across threads).
// Yh may be Xh (in place): each RHS chunk is staged before it is written.
template <typename R>
__global__ void __launch_bounds__(256) k_blockprod(const int2 *__restrict__ pairs, int npairs,
                                                   const cplx_t<R> *__restrict__ That,
                                                   const cplx_t<R> *Xh, cplx_t<R> *Yh, int b, int nrhs, int rch) {
    using C = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char zt_smem[];
    C *sT = reinterpret_cast<C *>(zt_smem);
    C *sf = sT + (size_t)b * b;
    C *sg = sf + (size_t)rch * b;
    const int rb = nrhs * b;
    for (int p = blockIdx.x; p < npairs; p += gridDim.x) {
        const int f = pairs[p].x, g = pairs[p].y;
        const C *Tb = That + (size_t)p * b * b;
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) sT[t] = Tb[t];
        for (int r0 = 0; r0 < nrhs; r0 += rch) {
            const int rc = min(rch, nrhs - r0);
            const int cb = rc * b;
            const C *xf = Xh + (size_t)f * rb + (size_t)r0 * b;
            const C *xg = Xh + (size_t)g * rb + (size_t)r0 * b;
            C *yf = Yh + (size_t)f * rb + (size_t)r0 * b;
            C *yg = Yh + (size_t)g * rb + (size_t)r0 * b;
            for (int t = threadIdx.x; t < cb; t += blockDim.x) {
                sf[t] = xf[t];
                if (g != f) sg[t] = xg[t];
            }
            __syncthreads();
            const int nout = (g != f ? 2 : 1) * cb;
            for (int o = threadIdx.x; o < nout; o += blockDim.x) {
                C acc = czero<C>();
                if (o < cb) {
                    const int rr = o / b, i = o - rr * b;
                    const C *row = sT + (size_t)i * b;
                    const C *xv = sf + (size_t)rr * b;
                    int j = i;
                    for (int jj = 0; jj < b; ++jj) {
                        acc = cfma(row[j], xv[j], acc);
                        if (++j == b) j = 0;
                    }
                    yf[o] = acc;
                } else {
                    const int o2 = o - cb;
                    const int rr = o2 / b, j = o2 - rr * b;
                    const C *xv = sg + (size_t)rr * b;
                    for (int i = 0; i < b; ++i) acc = cfma(sT[(size_t)i * b + j], xv[i], acc);
                    yg[o2] = acc;
                }
            }
            __syncthreads();
        }
    }
}

// Pipelined variant: persistent CTAs walk their pairs; for each pair the
// T^ block and the X^[f], X^[-f] slabs arrive by bulk async copies (TMA) into
// one of NST shared-memory stages, so NST pairs are in flight per CTA while
// the current one is multiplied.  Each output dot product may be split over S
// threads (S | b) so that every thread has work when 2 nrhs b < threads.
constexpr uint32_t kWaitTries = 1u << 22;  // bounded mbarrier waits
enum { ZT_ERRBIT_BLOCKPROD_WAIT = 1 };

template <typename R, int NST>
__global__ void __launch_bounds__(256) k_blockprod_tma(const int2 *__restrict__ pairs, int npairs,
                                                       const cplx_t<R> *__restrict__ That, cplx_t<R> *Xh, int b,
                                                       int nrhs, int S, int *err, cplx_t<R> *Yout, int l2hint) {
    using C = cplx_t<R>;
    extern __shared__ __align__(128) unsigned char zt_smem[];
    __shared__ __align__(8) uint64_t full[NST];
    __shared__ double2 red_raw[256];
    C *red = reinterpret_cast<C *>(red_raw);
    const int bb = b * b, rb = nrhs * b;
    const int stage_elems = bb + 2 * rb;
    C *stages = reinterpret_cast<C *>(zt_smem);
    const uint32_t tbytes = (uint32_t)(bb * sizeof(C)), xbytes = (uint32_t)(rb * sizeof(C));
    const int my = (npairs - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    uint64_t tpol = 0;
    if (threadIdx.x == 0 && l2hint) tpol = l2hint == 1 ? l2_policy_evict_last() : l2_policy_evict_first();
    auto issue = [&](int it) {  // thread 0
        const int p = blockIdx.x + it * gridDim.x;
        const int s = it % NST;
        const int2 fg = pairs[p];
        C *st = stages + (size_t)s * stage_elems;
        mbar_arrive_expect_tx(&full[s], tbytes + xbytes * (fg.y != fg.x ? 2u : 1u));
        if (l2hint)
            bulk_g2s_hint(st, That + (size_t)p * bb, tbytes, &full[s], tpol);
        else
            bulk_g2s(st, That + (size_t)p * bb, tbytes, &full[s]);
        bulk_g2s(st + bb, Xh + (size_t)fg.x * rb, xbytes, &full[s]);
        if (fg.y != fg.x) bulk_g2s(st + bb + rb, Xh + (size_t)fg.y * rb, xbytes, &full[s]);
    };
    if (threadIdx.x == 0)
        for (int it = 0; it < NST && it < my; ++it) issue(it);
    const int seg = b / S;
    for (int it = 0; it < my; ++it) {
        const int s = it % NST;
        const bool ok = mbar_wait_bounded(&full[s], (uint32_t)((it / NST) & 1), kWaitTries);
        if (__syncthreads_or(!ok)) {  // a copy never landed: record, drain what is in flight, leave
            if (threadIdx.x == 0) {
                atomicOr(err, ZT_ERRBIT_BLOCKPROD_WAIT);
                for (int k = it + 1; k < my && k < it + NST; ++k)
                    mbar_wait_bounded(&full[k % NST], (uint32_t)((k / NST) & 1), kWaitTries);
            }
            return;
        }
        const int p = blockIdx.x + it * gridDim.x;
        const int2 fg = pairs[p];
        const bool two = fg.y != fg.x;
        const C *T = stages + (size_t)s * stage_elems;
        const C *xf = T + bb, *xg = xf + rb;
        C *of = Yout + (size_t)fg.x * rb, *og = Yout + (size_t)fg.y * rb;
        const int nout = (two ? 2 : 1) * rb;
        if (S == 1) {
            for (int o = threadIdx.x; o < nout; o += blockDim.x) {
                C acc = czero<C>();
                if (o < rb) {
                    const int rr = o / b, i = o - rr * b;
                    const C *row = T + (size_t)i * b, *xv = xf + (size_t)rr * b;
                    int j = i;
                    for (int jj = 0; jj < b; ++jj) {
                        acc = cfma(row[j], xv[j], acc);
                        if (++j == b) j = 0;
                    }
                    of[o] = acc;
                } else {
                    const int o2 = o - rb, rr = o2 / b, j = o2 - rr * b;
                    const C *xv = xg + (size_t)rr * b;
                    for (int i = 0; i < b; ++i) acc = cfma(T[(size_t)i * b + j], xv[i], acc);
                    og[o2] = acc;
                }
            }
        } else {
            // outputs in chunks of opc, each dot split over S threads; the split
            // depends on b only, so a RHS is summed identically in any batch
            const int opc = blockDim.x / S;
            const int t = threadIdx.x, ol = t % opc, sp = t / opc;
            for (int ob = 0; ob < nout; ob += opc) {
                const int o = ob + ol;
                C acc = czero<C>();
                if (o < rb) {
                    const int rr = o / b, i = o - rr * b;
                    const C *row = T + (size_t)i * b, *xv = xf + (size_t)rr * b;
                    int j = i + sp * seg;
                    if (j >= b) j -= b;
                    for (int jj = 0; jj < seg; ++jj) {
                        acc = cfma(row[j], xv[j], acc);
                        if (++j == b) j = 0;
                    }
                } else if (o < nout) {
                    const int o2 = o - rb, rr = o2 / b, j = o2 - rr * b;
                    const C *xv = xg + (size_t)rr * b;
                    for (int i = sp * seg; i < (sp + 1) * seg; ++i) acc = cfma(T[(size_t)i * b + j], xv[i], acc);
                }
                red[sp * opc + ol] = acc;
                __syncthreads();
                if (sp == 0 && o < nout) {
                    C tot = red[ol];
                    for (int q = 1; q < S; ++q) tot = tot + red[q * opc + ol];
                    if (o < rb) of[o] = tot; else og[o - rb] = tot;
                }
                __syncthreads();
            }
        }
        __syncthreads();  // stage s is free again
        if (threadIdx.x == 0 && it + NST < my) issue(it + NST);
    }
}

// ------------------------------------------------------------ edge coupling
// One pass over B [E][ldb] (row e = edge unknown, column t = Toeplitz unknown)
// computing, for RHS r0..r0+RC-1,
//   ET[split][r][t] = sum_{e in split} B[e][t] x_E[r][e]     (B^T x_E)
//   Ep[tile][r][e]  = sum_{t in tile} B[e][t] x_T[r][t]       (B x_T partials)
// Each lane owns U 16-byte units of columns; B rows are read with fully
// coalesced 16-byte loads.  Row partials are reduced across the warp with
// shuffles and across warps through shared memory.
template <typename R> struct EdgeGeom {
    static constexpr int CPL = 16 / sizeof(cplx_t<R>);  // complex per 16-byte unit
    static constexpr int U = 2;                          // units per lane
    static constexpr int WARPS = 8;
    static constexpr int TILE = WARPS * 32 * U * CPL;    // columns per CTA
};

template <typename R>
__device__ __forceinline__ cplx_t<R> warp_sum(cplx_t<R> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

template <typename R>
__device__ __forceinline__ cplx_t<R> shfl_xor_c(cplx_t<R> v, int o) {
    v.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    return v;
}

// Warp reduce-scatter of 4 values: the result in lane l is the warp total of
// value ((l >> 4) & 1) * 2 + ((l >> 3) & 1).
template <typename R>
__device__ __forceinline__ cplx_t<R> warp_rs4(cplx_t<R> (&v)[4]) {
    const int lane = threadIdx.x & 31;
    const bool b4 = lane & 16, b3 = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const cplx_t<R> recv = shfl_xor_c<R>(b4 ? v[i] : v[i + 2], 16);
        v[i] = (b4 ? v[i + 2] : v[i]) + recv;
    }
    cplx_t<R> t = (b3 ? v[1] : v[0]) + shfl_xor_c<R>(b3 ? v[0] : v[1], 8);
    t = t + shfl_xor_c<R>(t, 4);
    t = t + shfl_xor_c<R>(t, 2);
    t = t + shfl_xor_c<R>(t, 1);
    return t;
}

template <typename R, int RC>
__global__ void __launch_bounds__(256) k_edge(const cplx_t<R> *__restrict__ x, const cplx_t<R> *__restrict__ B,
                                              cplx_t<R> *__restrict__ ET, cplx_t<R> *__restrict__ Ep,
                                              int64_t NT, int64_t ldb, int E, int64_t N, int nrhs, int r0,
                                              int rc, int e_per_split) {
    using C = cplx_t<R>;
    using G = EdgeGeom<R>;
    constexpr int CPL = G::CPL, U = G::U, W = G::WARPS;
    constexpr int CHUNK = 32;
    __shared__ C sxe[CHUNK][RC];
    __shared__ C red[W][CHUNK][RC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x, split = blockIdx.y;
    const int64_t tbase = (int64_t)tile * G::TILE + (int64_t)warp * (32 * U * CPL);
    const int e0 = split * e_per_split;
    const int e1 = min(E, e0 + e_per_split);

    C xt[U][CPL][RC];
    C acc[U][CPL][RC];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int64_t t = tbase + (int64_t)(u * 32 + lane) * CPL + c;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                acc[u][c][q] = czero<C>();
                xt[u][c][q] = (t < NT && q < rc) ? x[(int64_t)(r0 + q) * N + t] : czero<C>();
            }
        }

    for (int ec = e0; ec < e1; ec += CHUNK) {
        const int ne = min(CHUNK, e1 - ec);
        __syncthreads();
        for (int k = threadIdx.x; k < CHUNK * RC; k += blockDim.x) {
            const int el = k / RC, q = k - el * RC;
            sxe[el][q] = (el < ne && q < rc) ? x[(int64_t)(r0 + q) * N + NT + ec + el] : czero<C>();
        }
        __syncthreads();
        // Rows are consumed in groups of UNR whose loads are all issued first,
        // so each warp keeps UNR * 512 bytes of B in flight.
        constexpr int UNR = 4;
        for (int el0 = 0; el0 < ne; el0 += UNR) {
            float4 raw[UNR][U];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const C *brow = B + (int64_t)(ec + el0 + k) * ldb + tbase;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    raw[k][u] = (el0 + k < ne)
                                    ? __ldcs(reinterpret_cast<const float4 *>(brow + (int64_t)(u * 32 + lane) * CPL))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            C part[UNR][RC];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int el = el0 + k;
                C bv[U][CPL];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const C *pc = reinterpret_cast<const C *>(&raw[k][u]);
#pragma unroll
                    for (int c = 0; c < CPL; ++c) bv[u][c] = pc[c];
                }
#pragma unroll
                for (int q = 0; q < RC; ++q) {
                    const C xe = el < ne ? sxe[el][q] : czero<C>();  // padded rows hold zeros
                    C pt = czero<C>();
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int c = 0; c < CPL; ++c) {
                            if (el < ne) acc[u][c][q] = cfma(bv[u][c], xe, acc[u][c][q]);
                            pt = cfma(bv[u][c], xt[u][c][q], pt);
                        }
                    part[k][q] = pt;
                }
            }
            // reduce the 4 row partials across the warp at once: lane 8*k ends
            // with the total of row k (6 exchanges instead of 4 x 5)
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                C v4[UNR];
#pragma unroll
                for (int k = 0; k < UNR; ++k) v4[k] = part[k][q];
                const C tot = warp_rs4<R>(v4);
                const int k = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
                if ((lane & 7) == 0 && el0 + k < ne) red[warp][el0 + k][q] = tot;
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < ne * RC; k += blockDim.x) {
            const int el = k / RC, q = k - el * RC;
            if (q < rc) {
                C s = czero<C>();
#pragma unroll
                for (int w = 0; w < W; ++w) s = s + red[w][el][q];
                Ep[((int64_t)tile * nrhs + r0 + q) * E + ec + el] = s;
            }
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int64_t t = tbase + (int64_t)(u * 32 + lane) * CPL + c;
            if (t < NT) {
#pragma unroll
                for (int q = 0; q < RC; ++q)
                    if (q < rc) ET[((int64_t)split * nrhs + r0 + q) * NT + t] = acc[u][c][q];
            }
        }
}

// ET[0][r][t] += sum_{s >= 1} ET[s][r][t]: the B^T x_E rows in one buffer, so the
// inverse x pass reads a single value per output.
template <typename R>
__global__ void __launch_bounds__(256) k_fold_splits(cplx_t<R> *__restrict__ ET, int64_t count, int nsplit) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        cplx_t<R> s = ET[k];
        for (int sp = 1; sp < nsplit; ++sp) s = s + ET[(int64_t)sp * count + k];
        ET[k] = s;
    }
}

// y_E[r][e] = sum_tile Ep[tile][r][e] + sum_e' C[e][e'] x_E[r][e'].  One warp per (e, r).
template <typename R>
__global__ void __launch_bounds__(256) k_edge_finish(const cplx_t<R> *__restrict__ x, const cplx_t<R> *__restrict__ Cm,
                                                     const cplx_t<R> *__restrict__ Ep, cplx_t<R> *__restrict__ y,
                                                     int64_t NT, int E, int64_t N, int nrhs, int ntile) {
    using C = cplx_t<R>;
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int r = blockIdx.y;
    if (e >= E) return;
    C s = czero<C>();
    for (int t = lane; t < ntile; t += 32) s = s + Ep[((int64_t)t * nrhs + r) * E + e];
    const C *crow = Cm + (int64_t)e * E;
    const C *xe = x + (int64_t)r * N + NT;
    for (int k = lane; k < E; k += 32) s = cfma(crow[k], xe[k], s);
    s = warp_sum<R>(s);
    if (lane == 0) y[(int64_t)r * N + NT + e] = s;
}

// FP32 edge coupling in one pass over [B | C]: the FP32 copy of B carries C
// in the E columns after the N_T Toeplitz ones, so one row of it times the
// whole x = (x_T, x_E) is the edge row y_E = B x_T + C x_E.
//   ET[r][t]        = sum_e B[e][t] x_E[r][e]          (t < N_T; complete per column)
//   Ep[r][e][tile]  = sum_{t in tile} [B|C][e][t] x[r][t]  (row partials)
// A CTA owns a tile of E3_TW columns and reads all E rows of it; warp w takes
// rows w*UNR.., w*UNR + W*UNR.., ... (UNR rows per step, loads first), so each
// row's partial is one warp's and needs no cross-warp step; the B^T x_E sums
// of the warps are added in warp order through shared memory.  Rows are taken
// in chunks of E3_ECH so x_E fits in shared memory.  k_edge3_finish then adds
// each row's tile partials (the tile index is the fastest, so a warp reads a
// row's partials with coalesced loads) in a fixed order.
constexpr int E3_W = 8, E3_U = 2, E3_CPL = 2, E3_TW = 32 * E3_U * E3_CPL, E3_ECH = 1024;

template <int RC>
__global__ void __launch_bounds__(256) k_edge3(const float2 *__restrict__ x, const float2 *__restrict__ B,
                                               float2 *__restrict__ ET, float2 *__restrict__ Ep, int64_t NT,
                                               int64_t ncol, int64_t ldb, int E, int64_t N, int nrhs, int r0,
                                               int rc) {
    constexpr int U = E3_U, CPL = E3_CPL, W = E3_W, UNR = 4;
    // x_E of the current row chunk, later reused for the cross-warp sums
    constexpr int SX = E3_ECH * RC, SR = W * E3_TW * RC;
    __shared__ float2 sh[SX > SR ? SX : SR];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tile = blockIdx.x, ntile = gridDim.x;
    const int64_t tbase = (int64_t)tile * E3_TW;

    float2 xt[U][CPL][RC], acc[U][CPL][RC];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int64_t t = tbase + (int64_t)(u * 32 + lane) * CPL + c;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                acc[u][c][q] = make_float2(0.f, 0.f);
                xt[u][c][q] = (t < ncol && q < rc) ? x[(int64_t)(r0 + q) * N + t] : make_float2(0.f, 0.f);
            }
        }
    for (int ec = 0; ec < E; ec += E3_ECH) {
        const int ne = min(E3_ECH, E - ec);
        __syncthreads();
        for (int k = threadIdx.x; k < ne * RC; k += blockDim.x) {
            const int el = k / RC, q = k - el * RC;
            sh[k] = q < rc ? x[(int64_t)(r0 + q) * N + NT + ec + el] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int el0 = warp * UNR; el0 < ne; el0 += W * UNR) {
            float4 raw[UNR][U];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const float2 *brow = B + (int64_t)(ec + el0 + k) * ldb + tbase;
#pragma unroll
                for (int u = 0; u < U; ++u)
                    raw[k][u] = (el0 + k < ne)
                                    ? __ldcs(reinterpret_cast<const float4 *>(brow + (int64_t)(u * 32 + lane) * CPL))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            float2 part[UNR][RC];
#pragma unroll
            for (int k = 0; k < UNR; ++k) {
                const int el = el0 + k;
                float2 bv[U][CPL];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    bv[u][0] = make_float2(raw[k][u].x, raw[k][u].y);
                    bv[u][1] = make_float2(raw[k][u].z, raw[k][u].w);
                }
#pragma unroll
                for (int q = 0; q < RC; ++q) {
                    const float2 xe = el < ne ? sh[el * RC + q] : make_float2(0.f, 0.f);
                    float2 pt = make_float2(0.f, 0.f);
#pragma unroll
                    for (int u = 0; u < U; ++u)
#pragma unroll
                        for (int c = 0; c < CPL; ++c) {
                            acc[u][c][q] = cfma(bv[u][c], xe, acc[u][c][q]);
                            pt = cfma(bv[u][c], xt[u][c][q], pt);
                        }
                    part[k][q] = pt;
                }
            }
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                float2 v4[UNR];
#pragma unroll
                for (int k = 0; k < UNR; ++k) v4[k] = part[k][q];
                const float2 tot = warp_rs4<float>(v4);
                const int k = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
                if ((lane & 7) == 0 && el0 + k < ne && q < rc)
                    Ep[((int64_t)(r0 + q) * E + ec + el0 + k) * ntile + tile] = tot;
            }
        }
    }
    __syncthreads();
    // B^T x_E: add the W per-warp sums in warp order
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int q = 0; q < RC; ++q) sh[(warp * E3_TW + (u * 32 + lane) * CPL + c) * RC + q] = acc[u][c][q];
    __syncthreads();
    for (int k = threadIdx.x; k < E3_TW * RC; k += blockDim.x) {
        const int col = k / RC, q = k - col * RC;
        const int64_t t = tbase + col;
        if (t < NT && q < rc) {
            float2 sum = sh[col * RC + q];
#pragma unroll
            for (int w = 1; w < W; ++w) sum = sum + sh[(w * E3_TW + col) * RC + q];
            ET[(int64_t)(r0 + q) * NT + t] = sum;
        }
    }
}

// y[r][N_T + e] = sum_tile Ep[r][e][tile]: one warp per (r, e); lane l adds
// tiles l, l+32, ... in order (loads eight at a time), then a fixed
// butterfly over the lanes.
__global__ void __launch_bounds__(256) k_edge3_finish(const float2 *__restrict__ Ep, float2 *__restrict__ y,
                                                      int64_t NT, int E, int64_t N, int nrhs, int ntile) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // r * E + e
    if (row >= (int64_t)nrhs * E) return;
    const float2 *src = Ep + row * ntile;
    float2 s = make_float2(0.f, 0.f);
    int t = lane;
    for (; t + 7 * 32 < ntile; t += 8 * 32) {
        float2 v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __ldcg(src + t + i * 32);
#pragma unroll
        for (int i = 0; i < 8; ++i) s = s + v[i];
    }
    for (; t < ntile; t += 32) s = s + __ldcg(src + t);
    s = warp_sum<float>(s);
    if (lane == 0) {
        const int64_t r = row / E, e = row - r * E;
        y[r * N + NT + e] = s;
    }
}

// ------------------------------------------------------------ conversions
__global__ void k_c128_to_c64(const double2 *__restrict__ s, float2 *__restrict__ d, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        d[k] = make_float2((float)s[k].x, (float)s[k].y);
}
__global__ void k_c64_to_c128(const float2 *__restrict__ s, double2 *__restrict__ d, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        d[k] = make_double2(s[k].x, s[k].y);
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 32));
}

ztoep_status_t launch_c128_to_c64(const double2 *src, float2 *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return ZTOEP_OK;
    KScope ks(K_MISC, s);
    k_c128_to_c64<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}
ztoep_status_t launch_c64_to_c128(const float2 *src, double2 *dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return ZTOEP_OK;
    KScope ks(K_MISC, s);
    k_c64_to_c128<<<grid_for(n, 256), 256, 0, s>>>(src, dst, n);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// ------------------------------------------------------------ workspace
template <> MatvecWs &ws_of<float>(ztoep_plan_t p) { return p->ws32; }
template <> MatvecWs &ws_of<double>(ztoep_plan_t p) { return p->ws64; }

static int edge_ntile(ztoep_plan_t p, size_t csize) {
    int tile = (csize == 8) ? EdgeGeom<float>::TILE : EdgeGeom<double>::TILE;
    return (int)((p->NT + tile - 1) / tile);
}
// Tiles of k_edge3 over the N_T + E columns of [B | C].
static int edge3_ntile(ztoep_plan_t p) { return (int)((p->NT + p->E + E3_TW - 1) / E3_TW); }
static int edge_nsplit(ztoep_plan_t p, int ntile, size_t csize) {
    if (p->E == 0) return 0;
    // enough CTAs for several resident per SM (FP32: 4 per SM, FP64: 2)
    const int per_sm = csize == 8 ? 4 : 2;
    int want = (per_sm * p->nsm + ntile - 1) / ntile;
    int maxs = std::max(1, p->E / 32);
    return std::max(1, std::min(want, maxs));
}

// K chunk of the tensor-core B x_T product: enough (row tile, K split) CTAs to
// cover every SM twice, at least 256 complex k per CTA.
static int tc_edge_kchunk(ztoep_plan_t p) {
    if (p->tune.tc_kchunk > 0) return std::max(16, (p->tune.tc_kchunk + 15) / 16 * 16);
    const int mt = (p->E + 63) / 64;
    const int want = std::max(1, (2 * p->nsm + mt - 1) / mt);
    int kc = (int)((p->NT + want - 1) / want);
    kc = std::max(256, (kc + 15) / 16 * 16);
    return kc;
}
static int tc_edge_splits(ztoep_plan_t p) { return cgemm_splits((int)p->NT, tc_edge_kchunk(p)); }


static void free_ws(MatvecWs &w) {
    cudaFree(w.xin); cudaFree(w.yout); cudaFree(w.X1); cudaFree(w.Xh); cudaFree(w.ET); cudaFree(w.Ep); cudaFree(w.Yh);
    cudaFree(w.Ps); cudaFree(w.Us);
    w = MatvecWs{};
}

template <typename R> ztoep_status_t ensure_ws(ztoep_plan_t p, int nrhs) {
    MatvecWs &w = ws_of<R>(p);
    if (w.cap >= nrhs) return ZTOEP_OK;
    free_solve_graphs(p);
    free_ws(w);
    const size_t cs = sizeof(cplx_t<R>);
    const int ntile = edge_ntile(p, cs);
    const int nsplit = edge_nsplit(p, ntile, cs);
    size_t acc = 0;
    ZT_TRY(dalloc(&w.xin, cs * nrhs * p->N, &acc));
    ZT_TRY(dalloc(&w.yout, cs * nrhs * p->N, &acc));
    ZT_TRY(dalloc(&w.X1, cs * nrhs * (size_t)p->ny * p->lx * p->b, &acc));
    ZT_TRY(dalloc(&w.Xh, cs * nrhs * (size_t)p->F * p->b, &acc));
    const bool tc = cs == 8 && nrhs >= kTcMinRhs;
    if (p->E > 0 && p->side_k > 0) {  // side products: small frequency-domain buffers only
        ZT_TRY(dalloc(&w.Ps, cs * (size_t)nrhs * sides_partials(p), &acc));
        ZT_TRY(dalloc(&w.Us, cs * (size_t)4 * p->side_k * nrhs * std::max(p->lx, p->ly), &acc));
    } else if (p->E > 0) {
        ZT_TRY(dalloc(&w.ET, cs * (size_t)std::max(nsplit, 1) * nrhs * p->NT, &acc));
        const int parts = std::max(cs == 8 ? edge3_ntile(p) : ntile, tc ? tc_edge_splits(p) : 0);
        ZT_TRY(dalloc(&w.Ep, cs * (size_t)parts * nrhs * p->E, &acc));
    }
    if (tc || p->side_k > 0) ZT_TRY(dalloc(&w.Yh, cs * nrhs * (size_t)p->F * p->b, &acc));
    w.cap = nrhs;
    w.bytes = acc;
    return ZTOEP_OK;
}
template ztoep_status_t ensure_ws<float>(ztoep_plan_t, int);
template ztoep_status_t ensure_ws<double>(ztoep_plan_t, int);

template <typename R> static const cplx_t<R> *that_of(ztoep_plan_t p);
template <> const float2 *that_of<float>(ztoep_plan_t p) { return p->That32; }
template <> const double2 *that_of<double>(ztoep_plan_t p) { return p->That64; }
template <typename R> static const cplx_t<R> *b_of(ztoep_plan_t p);
template <> const float2 *b_of<float>(ztoep_plan_t p) { return p->B32; }
template <> const double2 *b_of<double>(ztoep_plan_t p) { return p->B64; }
template <typename R> static const cplx_t<R> *c_of(ztoep_plan_t p);
template <> const float2 *c_of<float>(ztoep_plan_t p) { return p->C32; }
template <> const double2 *c_of<double>(ztoep_plan_t p) { return p->C64; }
template <typename R> static const cplx_t<R> *twx_of(ztoep_plan_t p);
template <> const float2 *twx_of<float>(ztoep_plan_t p) { return p->twx32; }
template <> const double2 *twx_of<double>(ztoep_plan_t p) { return p->twx64; }
template <typename R> static const cplx_t<R> *twy_of(ztoep_plan_t p);
template <> const float2 *twy_of<float>(ztoep_plan_t p) { return p->twy32; }
template <> const double2 *twy_of<double>(ztoep_plan_t p) { return p->twy64; }

static int64_t edge_ldb(int64_t NT) { return (NT + 1023) / 1024 * 1024; }
// Row stride of the FP32 [B | C]: the N_T + E columns plus one sub-tile of
// zeros, so k_edge3's 16-byte loads of a sub-tile never leave the row.
static int64_t edge_ldb32(int64_t NT, int E) { return (NT + E + E3_TW + 1023) / 1024 * 1024; }

// Geometry of an FFT pass along dimension dim (0 = x, 1 = y): the heuristic,
// or the plan's tuned channel batch and thread count for FP32 passes (the
// batch clamped to what fits in shared memory).
static PassCfg plan_pass_cfg(ztoep_plan_t p, int dim, int L, int lines, size_t cs) {
    PassCfg c = pass_cfg(L, p->b, lines, cs, p->nsm);
    if (cs == 8) {
        if (p->tune.lib[dim] >= 0) c.lib = std::min(p->tune.lib[dim], pick_lib(L, p->b, cs, 64 * 1024));
        if (p->tune.thr[dim] > 0) c.threads = p->tune.thr[dim];
    }
    return c;
}

// FP32 pass kernel of dimension dim: the register kernel when the plan's
// choice and the length allow it.
static bool use_reg_pass(ztoep_plan_t p, int dim, int L) {
    return p->tune.fk[dim] != 1 && reg_fft_shape(L, nullptr);
}

// One FFT pass along dimension dim (0 = x, 1 = y) over `lines` lines per RHS:
// mk(ib) builds the load and store functors for a channel batch of ib.
template <typename R, bool INV, class MkLd, class MkSt>
static ztoep_status_t fft_pass(ztoep_plan_t p, int dim, int lines, int nrhs, const MkLd &mk_ld, const MkSt &mk_st,
                               cudaStream_t s) {
    const size_t cs = sizeof(cplx_t<R>);
    const int L = dim == 0 ? p->lx : p->ly;
    if constexpr (sizeof(cplx_t<R>) == 8) {
        if (use_reg_pass(p, dim, L)) {
            const int tuned = p->tune.lib[dim] >= 0 ? 1 << p->tune.lib[dim] : 0;
            const int cpb = reg_fft_cpb(L, p->b, lines * nrhs, p->nsm, tuned);
            const int ib = 2 * cpb;
            const dim3 g((p->b + ib - 1) / ib, lines, nrhs);
            return launch_fft_reg<INV>(L, dim == 0 ? p->twx32 : p->twy32, g, cpb, mk_ld(ib), mk_st(ib), s);
        }
    }
    const PassCfg c = plan_pass_cfg(p, dim, L, lines * nrhs, cs);
    const int ib = 1 << c.lib;
    const dim3 g((p->b + ib - 1) / ib, lines, nrhs);
    return launch_fft_pass<R>(dim == 0 ? p->fx : p->fy, dim == 0 ? twx_of<R>(p) : twy_of<R>(p), c.lib, INV, g,
                              mk_ld(ib), mk_st(ib), s, c.threads);
}

template <typename R>
static ztoep_status_t forward_passes(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *X1,
                                     cplx_t<R> *Xh, cudaStream_t s) {
    const uint8_t *act = p->masked ? p->active : nullptr;
    ZT_TRY((fft_pass<R, false>(
        p, 0, p->ny, nrhs, [&](int ib) { return LdXFwd<R>{x, act, p->nx, p->b, ib, p->N}; },
        [&](int ib) { return StX1<R>{X1, p->ny, p->lx, p->b, ib}; }, s)));
    ZT_TRY((fft_pass<R, false>(
        p, 1, p->lx, nrhs, [&](int ib) { return LdX1<R>{X1, p->ny, p->lx, p->b, ib}; },
        [&](int ib) { return StXh<R>{Xh, p->lx, p->b, ib, nrhs}; }, s)));
    return ZTOEP_OK;
}

// The pipelined (bulk-copy) block product applies: 16-byte multiples and two
// stages within 200 KB of shared memory.
template <typename R> static bool blockprod_pipelined(ztoep_plan_t p, int nrhs) {
    const size_t cs = sizeof(cplx_t<R>);
    const size_t tbytes = cs * (size_t)p->b * p->b, xbytes = cs * (size_t)nrhs * p->b;
    return tbytes % 16 == 0 && xbytes % 16 == 0 && 2 * (tbytes + 2 * xbytes) <= 200 * 1024;
}

// Block product on the pipelined kernel when it applies, else the staged
// fallback; `out` (default Xh: in place) receives Y^.
template <typename R>
static ztoep_status_t launch_blockprod(ztoep_plan_t p, int nrhs, cplx_t<R> *Xh, cudaStream_t s,
                                       cplx_t<R> *out = nullptr) {
    if (!out) out = Xh;
    const size_t cs = sizeof(cplx_t<R>);
    const size_t budget = 200 * 1024;
    const size_t tbytes = cs * (size_t)p->b * p->b;
    const size_t xbytes = cs * (size_t)nrhs * p->b;
    const size_t stage = tbytes + 2 * xbytes;
    KScope ks(K_BLOCKPROD, s);
    if (tbytes % 16 == 0 && xbytes % 16 == 0 && 2 * stage <= budget) {
        // pipelined bulk-copy path
        const int nst = 3 * stage <= budget ? 3 : 2;
        const size_t smem = nst * stage;
        const int fit = std::max<int>(1, std::min<int>(4, (int)((227 * 1024) / (smem + 6 * 1024))));
        const int per_sm = p->tune.bp_per_sm > 0 ? std::min(p->tune.bp_per_sm, fit) : fit;
        const int grid = std::min(p->npairs, p->nsm * per_sm);
        int S = 1;  // threads per dot product: from b (or the plan's choice) only, batch-independent sums
        if (p->tune.bp_split > 0 && p->b % p->tune.bp_split == 0 && p->tune.bp_split <= 8) {
            S = p->tune.bp_split;
        } else {
            for (int c : {8, 4, 2})
                if (p->b % c == 0 && c * 2 * p->b <= 256) { S = c; break; }
        }
        static bool attr = false;
        if (!attr) {
            ZT_CUDA(cudaFuncSetAttribute(k_blockprod_tma<R, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
            ZT_CUDA(cudaFuncSetAttribute(k_blockprod_tma<R, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
            attr = true;
        }
        // The spectrum is re-read by every product: kept in L2 (evict_last)
        // when it takes at most 3/4 of it, streamed (evict_first) when it is
        // over twice its size, so the vectors stay cached instead.
        const size_t spec = (size_t)p->npairs * tbytes, l2 = (size_t)std::max(p->l2_bytes, 0);
        const int l2hint = l2 == 0 ? 0 : (4 * spec <= 3 * l2 ? 1 : (spec > 2 * l2 ? 2 : 0));
        if (nst == 3)
            k_blockprod_tma<R, 3><<<grid, 256, smem, s>>>(p->pairs, p->npairs, that_of<R>(p), Xh, p->b, nrhs, S, p->err,
                                                          out, l2hint);
        else
            k_blockprod_tma<R, 2><<<grid, 256, smem, s>>>(p->pairs, p->npairs, that_of<R>(p), Xh, p->b, nrhs, S, p->err,
                                                          out, l2hint);
        ZT_CUDA(cudaGetLastError());
        return ZTOEP_OK;
    }
    if (tbytes + 2 * cs * p->b > budget) return ZTOEP_ERR_UNSUPPORTED;
    const int rch = (int)std::min<size_t>((size_t)nrhs, (budget - tbytes) / (2 * cs * p->b));
    const size_t smem = tbytes + 2 * cs * (size_t)rch * p->b;
    static bool attr = false;
    if (!attr) {
        ZT_CUDA(cudaFuncSetAttribute(k_blockprod<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr = true;
    }
    k_blockprod<R><<<p->npairs, 256, smem, s>>>(p->pairs, p->npairs, that_of<R>(p), Xh, out, p->b, nrhs, rch);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

template <typename R>
static ztoep_status_t launch_edge(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *y,
                                  MatvecWs &w, cudaStream_t s, bool fold = false) {
    const size_t cs = sizeof(cplx_t<R>);
    const int ntile = edge_ntile(p, cs);
    const int nsplit = edge_nsplit(p, ntile, cs);
    const int eps = (p->E + nsplit - 1) / nsplit;
    cplx_t<R> *ET = reinterpret_cast<cplx_t<R> *>(w.ET);
    cplx_t<R> *Ep = reinterpret_cast<cplx_t<R> *>(w.Ep);
    const int64_t ldb = edge_ldb(p->NT);
    for (int r0 = 0; r0 < nrhs; r0 += 4) {
        const int rc = std::min(4, nrhs - r0);
        dim3 g(ntile, nsplit);
        KScope ks(K_EDGE, s);
        if (rc == 1)
            k_edge<R, 1><<<g, 256, 0, s>>>(x, b_of<R>(p), ET, Ep, p->NT, ldb, p->E, p->N, nrhs, r0, rc, eps);
        else if (rc == 2)
            k_edge<R, 2><<<g, 256, 0, s>>>(x, b_of<R>(p), ET, Ep, p->NT, ldb, p->E, p->N, nrhs, r0, rc, eps);
        else
            k_edge<R, 4><<<g, 256, 0, s>>>(x, b_of<R>(p), ET, Ep, p->NT, ldb, p->E, p->N, nrhs, r0, rc, eps);
        ZT_CUDA(cudaGetLastError());
    }
    dim3 gf((p->E + 7) / 8, nrhs);
    KScope ks(K_MISC, s);
    ks.add(fold && nsplit > 1 ? 2 : 1);
    k_edge_finish<R><<<gf, 256, 0, s>>>(x, c_of<R>(p), Ep, y, p->NT, p->E, p->N, nrhs, ntile);
    if (fold && nsplit > 1) {
        const int64_t count = (int64_t)nrhs * p->NT;
        k_fold_splits<R><<<grid_for(count, 256), 256, 0, s>>>(ET, count, nsplit);
    }
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// FP32 edge coupling (k_edge3, then k_edge3_finish): ET holds B^T x_E and
// y_E = B x_T + C x_E.  et_ready is recorded once ET is final (the finish
// only writes y_E).
static ztoep_status_t launch_edge3(ztoep_plan_t p, int nrhs, const float2 *x, float2 *y, MatvecWs &w,
                                   cudaStream_t s, cudaEvent_t et_ready) {
    float2 *ET = reinterpret_cast<float2 *>(w.ET);
    float2 *Ep = reinterpret_cast<float2 *>(w.Ep);
    const int ntile = edge3_ntile(p);
    const int64_t ldb = edge_ldb32(p->NT, p->E), ncol = p->NT + p->E;
    for (int r0 = 0; r0 < nrhs; r0 += 4) {
        const int rc = std::min(4, nrhs - r0);
        KScope ks(K_EDGE, s);
        if (rc == 1)
            k_edge3<1><<<ntile, 256, 0, s>>>(x, p->B32, ET, Ep, p->NT, ncol, ldb, p->E, p->N, nrhs, r0, rc);
        else if (rc == 2)
            k_edge3<2><<<ntile, 256, 0, s>>>(x, p->B32, ET, Ep, p->NT, ncol, ldb, p->E, p->N, nrhs, r0, rc);
        else
            k_edge3<4><<<ntile, 256, 0, s>>>(x, p->B32, ET, Ep, p->NT, ncol, ldb, p->E, p->N, nrhs, r0, rc);
        ZT_CUDA(cudaGetLastError());
    }
    if (et_ready) ZT_CUDA(cudaEventRecord(et_ready, s));
    KScope ks(K_MISC, s);
    const int64_t rows = (int64_t)nrhs * p->E;
    k_edge3_finish<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(Ep, y, p->NT, p->E, p->N, nrhs, ntile);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// Tensor-core edge coupling (FP32 products, kTcMinRhs..kTcMaxRhs RHS):
//   B x_T    as C[e][q] = sum_t B[e][t] x_T[q][t]   -> K-split partials in Ep
//   B^T x_E  as C[t][q] = sum_e B^T[t][e] x_E[q][e] -> ET[0]
// then y_E = sum of the partials + C x_E.
static ztoep_status_t tc_edge(ztoep_plan_t p, int nrhs, const float2 *x, float2 *y, MatvecWs &w, cudaStream_t s,
                              cudaEvent_t et_ready = nullptr) {
    const int kc = tc_edge_kchunk(p);
    CgemmArgs g1{};
    g1.A = p->B32; g1.lda = edge_ldb32(p->NT, p->E); g1.strideA = 0;
    g1.X = x; g1.ldx = p->N; g1.strideX = 0;
    g1.C = reinterpret_cast<float2 *>(w.Ep); g1.ldc_q = p->E; g1.ldc_m = 1; g1.strideC = 0;
    g1.strideCk = (int64_t)nrhs * p->E;
    g1.M = p->E; g1.K = (int)p->NT; g1.N = nrhs; g1.kchunk = kc; g1.err = p->err;
    ZT_TRY(launch_cgemm(g1, 1, p->nsm, s));
    CgemmArgs g2{};
    g2.A = p->B32T; g2.lda = p->E; g2.strideA = 0;
    g2.X = x + p->NT; g2.ldx = p->N; g2.strideX = 0;
    g2.C = reinterpret_cast<float2 *>(w.ET); g2.ldc_q = p->NT; g2.ldc_m = 1; g2.strideC = 0; g2.strideCk = 0;
    g2.M = (int)p->NT; g2.K = p->E; g2.N = nrhs; g2.kchunk = 0; g2.err = p->err;
    ZT_TRY(launch_cgemm(g2, 1, p->nsm, s));
    if (et_ready) ZT_CUDA(cudaEventRecord(et_ready, s));  // ET is final; the finish only writes y_E
    dim3 gf((p->E + 7) / 8, nrhs);
    KScope ks(K_MISC, s);
    k_edge_finish<float><<<gf, 256, 0, s>>>(x, p->C32, reinterpret_cast<const float2 *>(w.Ep), y, p->NT, p->E,
                                            p->N, nrhs, cgemm_splits((int)p->NT, kc));
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// Tensor-core block product: Yh[f] = T^[f] Xh[f] for every frequency (full
// FP32 spectrum, separate output buffer).
static ztoep_status_t tc_blockprod(ztoep_plan_t p, int nrhs, const float2 *Xh, float2 *Yh, cudaStream_t s) {
    CgemmArgs g{};
    g.A = p->That32full; g.lda = p->b; g.strideA = (int64_t)p->b * p->b;
    g.X = Xh; g.ldx = p->b; g.strideX = (int64_t)nrhs * p->b;
    g.C = Yh; g.ldc_q = p->b; g.ldc_m = 1; g.strideC = (int64_t)nrhs * p->b; g.strideCk = 0;
    g.M = p->b; g.K = p->b; g.N = nrhs; g.kchunk = 0; g.err = p->err;
    return launch_cgemm(g, p->F, p->nsm, s);
}

template <typename R> static bool use_tensor(ztoep_plan_t p, int nrhs) {
    if (sizeof(R) != sizeof(float) || nrhs < kTcMinRhs || nrhs > kTcMaxRhs || !cgemm_fits(nrhs)) return false;
    return p->That32full != nullptr && (p->E == 0 || p->side_k > 0 || p->B32T != nullptr);
}

// Stream of the product's concurrent branch: the plan's second stream, or the
// launching stream itself while instrumentation asks for serial branches
// (outside graph captures).
static cudaStream_t branch_stream(ztoep_plan_t p, cudaStream_t s) {
    if (!timing_serial()) return p->side;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    return cs == cudaStreamCaptureStatusNone ? s : p->side;
}

template <typename R>
ztoep_status_t run_matvec(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *y, cudaStream_t s) {
    ZT_TRY(ensure_ws<R>(p, nrhs));
    MatvecWs &w = ws_of<R>(p);
    const size_t cs = sizeof(cplx_t<R>);
    cplx_t<R> *X1 = reinterpret_cast<cplx_t<R> *>(w.X1);
    cplx_t<R> *Xh = reinterpret_cast<cplx_t<R> *>(w.Xh);
    const int ntile = edge_ntile(p, cs);
    const int nsplit = p->side_k > 0 ? 0 : edge_nsplit(p, ntile, cs);
    const bool tc = use_tensor<R>(p, nrhs) && w.Yh != nullptr;
    const bool sides = p->E > 0 && p->side_k > 0;
    const cudaStream_t br = branch_stream(p, s);
    if (p->E > 0 && !sides) {  // edge branch on the side stream, concurrent with the FFT chain
        ZT_CUDA(cudaEventRecord(p->ev_fork, s));
        ZT_CUDA(cudaStreamWaitEvent(br, p->ev_fork, 0));
        if (tc) {
            ZT_TRY(tc_edge(p, nrhs, reinterpret_cast<const float2 *>(x), reinterpret_cast<float2 *>(y), w, br,
                           p->ev_et));
        } else if (sizeof(R) == sizeof(float)) {
            ZT_TRY(launch_edge3(p, nrhs, reinterpret_cast<const float2 *>(x), reinterpret_cast<float2 *>(y), w, br,
                                p->ev_et));
        } else {
            ZT_TRY(launch_edge<R>(p, nrhs, x, y, w, br, true));
            ZT_CUDA(cudaEventRecord(p->ev_et, br));
        }
        ZT_CUDA(cudaEventRecord(p->ev_join, br));
    } else if (sides) {  // side stream: the DFTs of the side slices of x_E beside the forward passes
        ZT_CUDA(cudaEventRecord(p->ev_fork, s));
        ZT_CUDA(cudaStreamWaitEvent(br, p->ev_fork, 0));
        ZT_TRY(sides_uhat<R>(p, nrhs, x, w, br));
        ZT_CUDA(cudaEventRecord(p->ev_et, br));
    }
    ZT_TRY(forward_passes<R>(p, nrhs, x, X1, Xh, s));
    cplx_t<R> *Yh = Xh;
    if (sides) {
        // block product out of place (X^ stays for B x_T), both side products
        // in one pass over the generator spectra, then y_E on the side stream
        // beside the inverse passes
        Yh = reinterpret_cast<cplx_t<R> *>(w.Yh);
        if (tc)
            ZT_TRY(tc_blockprod(p, nrhs, reinterpret_cast<const float2 *>(Xh), reinterpret_cast<float2 *>(Yh), s));
        else
            ZT_TRY(launch_blockprod<R>(p, nrhs, Xh, s, Yh));
        ZT_CUDA(cudaStreamWaitEvent(s, p->ev_et, 0));  // U from the side stream
        ZT_TRY(sides_fused<R>(p, nrhs, Xh, Yh, w, s));
        ZT_CUDA(cudaEventRecord(p->ev_fork, s));
        ZT_CUDA(cudaStreamWaitEvent(br, p->ev_fork, 0));
        ZT_TRY(sides_finish<R>(p, nrhs, x, y, w, br));
        ZT_CUDA(cudaEventRecord(p->ev_join, br));
    } else if (tc) {
        Yh = reinterpret_cast<cplx_t<R> *>(w.Yh);
        ZT_TRY(tc_blockprod(p, nrhs, reinterpret_cast<const float2 *>(Xh), reinterpret_cast<float2 *>(Yh), s));
    } else {
        ZT_TRY(launch_blockprod<R>(p, nrhs, Xh, s));
    }
    ZT_TRY((fft_pass<R, true>(
        p, 1, p->lx, nrhs, [&](int ib) { return LdXh<R>{Yh, p->lx, p->b, ib, nrhs}; },
        [&](int ib) { return StY1<R>{X1, p->ny, p->lx, p->b, ib}; }, s)));
    // the last pass adds B^T x_E (dense B): it waits for that term only; the
    // edge rows y_E (and the side branch) are joined at the end
    if (p->E > 0 && !sides) ZT_CUDA(cudaStreamWaitEvent(s, p->ev_et, 0));
    const R scale = (R)(1.0 / ((double)p->lx * (double)p->ly));
    const cplx_t<R> *ET = reinterpret_cast<const cplx_t<R> *>(w.ET);
    const uint8_t *act = p->masked ? p->active : nullptr;
    const int ns = nsplit > 0 ? 1 : 0;
    ZT_TRY((fft_pass<R, true>(
        p, 0, p->ny, nrhs, [&](int ib) { return LdY1<R>{X1, p->ny, p->lx, p->b, ib}; },
        [&](int ib) {
            return StYOut<R>{y, x, ET, act, p->nx, p->b, ib, nrhs, ns, p->N, p->NT, scale};
        },
        s)));
    if (p->E > 0) ZT_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
    return ZTOEP_OK;
}
template ztoep_status_t run_matvec<float>(ztoep_plan_t, int, const float2 *, float2 *, cudaStream_t);
template ztoep_status_t run_matvec<double>(ztoep_plan_t, int, const double2 *, double2 *, cudaStream_t);

template <typename R>
ztoep_status_t run_forward_spectrum(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *Xh,
                                    cudaStream_t s) {
    ZT_TRY(ensure_ws<R>(p, nrhs));
    MatvecWs &w = ws_of<R>(p);
    return forward_passes<R>(p, nrhs, x, reinterpret_cast<cplx_t<R> *>(w.X1), Xh, s);
}
template ztoep_status_t run_forward_spectrum<float>(ztoep_plan_t, int, const float2 *, float2 *, cudaStream_t);
template ztoep_status_t run_forward_spectrum<double>(ztoep_plan_t, int, const double2 *, double2 *, cudaStream_t);

void free_matvec_ws(ztoep_plan_t p) {
    free_ws(p->ws32);
    free_ws(p->ws64);
}

int64_t edge_row_stride(int64_t NT) { return edge_ldb(NT); }
int64_t edge_row_stride32(int64_t NT, int E) { return edge_ldb32(NT, E); }

// [B | C] in FP32 from the FP64 B (row stride ldb64) and C: row e holds
// B[e][0..NT), C[e][0..E), then zeros up to ldb32.
__global__ void k_pack_bc32(const double2 *__restrict__ B, int64_t ldb64, const double2 *__restrict__ Cm,
                            float2 *__restrict__ out, int64_t ldb32, int E, int64_t NT) {
    const int64_t total = (int64_t)E * ldb32;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = k / ldb32, t = k - e * ldb32;
        double2 v = make_double2(0.0, 0.0);
        if (t < NT)
            v = B[e * ldb64 + t];
        else if (t < NT + E)
            v = Cm[e * (int64_t)E + (t - NT)];
        out[k] = make_float2((float)v.x, (float)v.y);
    }
}

ztoep_status_t pack_bc32(ztoep_plan_t p, cudaStream_t s) {
    KScope ks(K_MISC, s);
    k_pack_bc32<<<1024, 256, 0, s>>>(p->B64, edge_ldb(p->NT), p->C64, p->B32, edge_ldb32(p->NT, p->E), p->E, p->NT);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

}  // namespace ztoep

// ------------------------------------------------------------ tensor-core operands
namespace ztoep {

// Full FP32 spectrum: block of -f is the transpose of the stored block of f.
__global__ void k_expand_spectrum32(const float2 *__restrict__ T32, const int *__restrict__ rep, float2 *out, int F,
                                    int b) {
    const int64_t bb = (int64_t)b * b;
    const int64_t total = (int64_t)F * bb;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        const int f = (int)(k / bb);
        const int64_t c = k - f * bb;
        const int i = (int)(c / b), j = (int)(c - (int64_t)i * b);
        const int r = rep[f];
        out[k] = r >= 0 ? T32[(int64_t)r * bb + c] : T32[(int64_t)(-1 - r) * bb + (int64_t)j * b + i];
    }
}

// BT[t][e] = B[e][t] through 32 x 32 shared-memory tiles.
__global__ void k_transpose32(const float2 *__restrict__ B, int64_t ldb, float2 *__restrict__ BT, int E, int64_t NT) {
    __shared__ float2 tile[32][33];
    const int64_t t0 = (int64_t)blockIdx.x * 32;
    const int e0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int e = e0 + r;
        const int64_t t = t0 + threadIdx.x;
        tile[r][threadIdx.x] = (e < E && t < NT) ? B[(int64_t)e * ldb + t] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t t = t0 + r;
        const int e = e0 + threadIdx.x;
        if (t < NT && e < E) BT[t * E + e] = tile[threadIdx.x][r];
    }
}

ztoep_status_t ensure_tensor_data(ztoep_plan_t p, int nrhs, cudaStream_t s) {
    if (nrhs < kTcMinRhs || nrhs > kTcMaxRhs) return ZTOEP_OK;
    size_t acc = 0;
    if (!p->That32full) {
        ZT_TRY(dalloc((void **)&p->That32full, sizeof(float2) * (size_t)p->F * p->b * p->b, &acc));
        KScope ks(K_MISC, s);
        k_expand_spectrum32<<<1024, 256, 0, s>>>(p->That32, p->rep, p->That32full, p->F, p->b);
        ZT_CUDA(cudaGetLastError());
    }
    if (p->E > 0 && p->side_k == 0 && !p->B32T) {
        ZT_TRY(dalloc((void **)&p->B32T, sizeof(float2) * (size_t)p->NT * p->E, &acc));
        dim3 g((unsigned)((p->NT + 31) / 32), (unsigned)((p->E + 31) / 32));
        KScope ks(K_MISC, s);
        k_transpose32<<<g, dim3(32, 8), 0, s>>>(p->B32, edge_ldb32(p->NT, p->E), p->B32T, p->E, p->NT);
        ZT_CUDA(cudaGetLastError());
    }
    p->tc_bytes += acc;
    return ZTOEP_OK;
}

}  // namespace ztoep

// ------------------------------------------------------------ allocation-free edge product
// Some callers cannot allocate device memory when they call into the library:
// real-time or embedded hosts that forbid allocation after start-up (an
// allocation can block for a device-wide synchronisation or fail under
// fragmentation at an unpredictable moment), and frameworks whose memory pool
// has already reserved every device byte, so that a cudaMalloc of ours would
// fail or evict their cache.
// For them ztoep_edge_product_noalloc computes the edge-coupling part of the
// FP64 product with its partial sums in the fixed array below instead of the
// plan's lazily allocated workspace.  The array is 16 MiB, lives on every
// device that loads this library until the process exits, is shared by all
// calls (so two calls whose work overlaps on the GPU race on it) and keeps
// whatever the last call left in it; every call overwrites all the scratch it
// reads, so nothing in it has to start at zero.
namespace ztoep {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static void *g_noalloc_addr[kMaxDevices];
static std::mutex g_noalloc_mu;

// Device address of g_noalloc_scratch on the current device, looked up once
// per device (host code only sees a host-side stand-in for the symbol).
static ztoep_status_t noalloc_scratch(int dev, void **out) {
    if (dev < 0 || dev >= kMaxDevices) return ZTOEP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return ZTOEP_ERR_CUDA;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return ZTOEP_OK;
}

// y[r][t] = sum_s ET[s][r][t] (the B^T x_E rows), t < NT.
__global__ void k_sum_splits(const double2 *__restrict__ ET, double2 *__restrict__ y, int64_t NT, int64_t N,
                             int nrhs, int nsplit) {
    const int64_t total = (int64_t)nrhs * NT;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = k / NT, t = k - r * NT;
        double2 s = ET[k];
        for (int sp = 1; sp < nsplit; ++sp) s = s + ET[(int64_t)sp * total + k];
        y[r * N + t] = s;
    }
}

static size_t round256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace ztoep

extern "C" ztoep_status_t ztoep_edge_product_noalloc(ztoep_plan_t p, int32_t nrhs, const void *X, void *Y,
                                                     void *stream) {
    using namespace ztoep;
    if (!p || !X || !Y || nrhs < 1) return ZTOEP_ERR_ARG;
    const size_t vbytes = sizeof(double2) * (size_t)nrhs * p->N;
    if (bytes_overlap(X, vbytes, Y, vbytes)) return ZTOEP_ERR_ARG;
    int dev = -1;
    ZT_CUDA(cudaGetDevice(&dev));
    if (dev != p->device) return ZTOEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double2 *y = (double2 *)Y;
    const double2 *x = (const double2 *)X;
    if (p->side_k > 0) return ZTOEP_ERR_UNSUPPORTED;  // no dense B kept: use ztoep_matvec
    if (p->E == 0) {  // no edge unknowns: the edge part of the product is zero
        ZT_CUDA(cudaMemsetAsync(y, 0, sizeof(double2) * (size_t)nrhs * p->N, s));
        return ZTOEP_OK;
    }
    const int ntile = edge_ntile(p, sizeof(double2));
    const int nsplit = edge_nsplit(p, ntile, sizeof(double2));
    const size_t et_bytes = round256(sizeof(double2) * (size_t)nsplit * nrhs * p->NT);
    const size_t ep_bytes = round256(sizeof(double2) * (size_t)ntile * nrhs * p->E);
    if (et_bytes + ep_bytes > kNoAllocScratchBytes) return ZTOEP_ERR_NOMEM;
    void *base = nullptr;
    ZT_TRY(noalloc_scratch(dev, &base));
    MatvecWs w{};  // views into the fixed scratch; owns nothing
    w.ET = base;
    w.Ep = (unsigned char *)base + et_bytes;
    std::lock_guard<std::mutex> lk(p->mu);
    ZT_TRY(launch_edge<double>(p, nrhs, x, y, w, s));
    KScope ks(K_MISC, s);
    k_sum_splits<<<grid_for((int64_t)nrhs * p->NT, 256), 256, 0, s>>>((const double2 *)w.ET, y, p->NT, p->N,
                                                                      nrhs, nsplit);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}
