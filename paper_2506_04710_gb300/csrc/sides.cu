// Structured edge coupling: perimeter edge unknowns whose side blocks of B are
// one-level block Toeplitz along the side (Sec. II-C, the side blocks of
// Eqs. submatrixB12/B34).
//
// Layout (k edge unknowns per cell side, counter-clockwise from (0, 0)): side
// 0 bottom (cells c = m, left to right), 1 right (c = n, upwards), 2 top
// (c = m, unknowns stored right to left), 3 left (c = n, stored downwards);
// within a cell the sub-position s runs along the side's positive direction.
// The entry of edge unknown (side, c, s) and Toeplitz unknown (m, n, i) is a
// generator value g[side][s][p][o][i] with p = c - m, o = n on the bottom and
// top sides and p = c - n, o = m on the right and left sides.
//
// Each generator is embedded in the Ly x Lx grid of the 2-D circulant
// embedding (bottom/top: row o, column p mod Lx; right/left: row p mod Ly,
// column o) and transformed once at plan time, G^.  With X^, Y^ the 2-D
// spectra of the FFT product (unnormalised DFT, exp(-2 pi i k n / L)):
//   B x_T, bottom/top: F(kx) = sum_{ky,i} G^[ky][kx][i] X^[-ky][kx][i],
//                      y_E(c) = 1/(Lx Ly) sum_kx exp(+2 pi i kx c / Lx) F(kx)
//   B x_T, right/left: F(ky) = sum_{kx,i} G^[ky][kx][i] X^[ky][-kx][i], likewise over ky
//   B^T x_E:           Y^[ky][kx][i] += sum_s G^[ky][-kx][i] U_s(kx)   (bottom/top)
//                      Y^[ky][kx][i] += sum_s G^[-ky][kx][i] U_s(ky)   (right/left)
//                      with U_s(k) = sum_c x_E(side, c, s) exp(-2 pi i k c / L),
// and the inverse passes of the product apply the 1/(Lx Ly).  The embedding
// sizes Lx >= 2Nx - 1, Ly >= 2Ny - 1 of the block product keep these
// convolutions free of wrap-around, so the results equal the dense products.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "instrument.cuh"
#include "tma.cuh"

namespace ztoep {

namespace {

struct SideMap {
    int nx, ny, k;
    __host__ __device__ int len(int sg) const { return (sg & 1) ? ny : nx; }
    __host__ __device__ int base(int sg) const {
        return sg == 0 ? 0 : sg == 1 ? k * nx : sg == 2 ? k * (nx + ny) : k * (2 * nx + ny);
    }
    __host__ __device__ int edge(int sg, int c, int s) const {
        return sg < 2 ? base(sg) + k * c + s : base(sg) + k * (len(sg) - 1 - c) + (k - 1 - s);
    }
    __host__ __device__ void locate(int e, int &sg, int &c, int &s) const {
        sg = e < base(1) ? 0 : e < base(2) ? 1 : e < base(3) ? 2 : 3;
        const int j = e - base(sg), q = j / k, r = j - q * k;
        if (sg < 2) {
            c = q;
            s = r;
        } else {
            c = len(sg) - 1 - q;
            s = k - 1 - r;
        }
    }
};

// RHS per block of the fused side kernel, and RHS per step (registers).
template <typename R> constexpr int side_rb() { return sizeof(R) == sizeof(float) ? 8 : 4; }
template <typename R> constexpr int side_rq(int nv) { return sizeof(R) == sizeof(float) || nv < 16 ? 2 : 1; }
// FP32: the next row's G^ is copied into shared memory while a row is
// computed; FP64 loads it directly (two stages would take one SM's memory).
template <typename R> constexpr bool side_prefetch() { return sizeof(R) == sizeof(float); }

// Embedded generator grids G[(side*k + s)][y][x][i] (FP64), read from B.
__global__ void k_side_embed(const double2 *__restrict__ B, double2 *__restrict__ G, SideMap sm, int b, int lx,
                             int ly, int64_t NT) {
    const int64_t per = (int64_t)ly * lx * b;
    const int64_t total = per * 4 * sm.k;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int gs = (int)(idx / per);
        int64_t rem = idx - gs * per;
        const int y = (int)(rem / ((int64_t)lx * b));
        rem -= (int64_t)y * lx * b;
        const int x = (int)(rem / b), i = (int)(rem - (int64_t)x * b);
        const int sg = gs / sm.k, s = gs - sg * sm.k;
        double2 v = make_double2(0.0, 0.0);
        if ((sg & 1) == 0) {  // bottom / top: row o = n, column p mod lx
            const int p = x < sm.nx ? x : x - lx;
            if (y < sm.ny && p > -sm.nx && p < sm.nx) {
                const int c = p > 0 ? p : 0, m = c - p;
                v = B[(int64_t)sm.edge(sg, c, s) * NT + ((int64_t)y * sm.nx + m) * b + i];
            }
        } else {  // right / left: row p mod ly, column o = m
            const int p = y < sm.ny ? y : y - ly;
            if (x < sm.nx && p > -sm.ny && p < sm.ny) {
                const int c = p > 0 ? p : 0, n = c - p;
                v = B[(int64_t)sm.edge(sg, c, s) * NT + ((int64_t)n * sm.nx + x) * b + i];
            }
        }
        G[idx] = v;
    }
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double v) {
    atomicMax(a, (unsigned long long)__double_as_longlong(v));  // non-negative doubles order as their bits
}

// max |B[e][t] - generator value| and max |B[e][t]| over all e and all t.
__global__ void k_side_verify(const double2 *__restrict__ B, const double2 *__restrict__ G, SideMap sm, int b,
                              int lx, int ly, int64_t NT, int E, unsigned long long *out) {
    __shared__ double red[2][8];
    double dmax = 0.0, bmax = 0.0;
    const int64_t total = (int64_t)E * NT;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)(idx / NT);
        const int64_t t = idx - (int64_t)e * NT;
        const int el = (int)(t / b), i = (int)(t - (int64_t)el * b);
        const int n = el / sm.nx, m = el - n * sm.nx;
        int sg, c, s;
        sm.locate(e, sg, c, s);
        int y, x;
        if ((sg & 1) == 0) {
            const int p = c - m;
            y = n;
            x = p >= 0 ? p : p + lx;
        } else {
            const int p = c - n;
            y = p >= 0 ? p : p + ly;
            x = m;
        }
        const double2 bv = B[idx];
        const double2 gv = G[((((int64_t)(sg * sm.k + s) * ly + y) * lx) + x) * b + i];
        dmax = fmax(dmax, hypot(bv.x - gv.x, bv.y - gv.y));
        bmax = fmax(bmax, hypot(bv.x, bv.y));
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = dmax;
        red[1][w] = bmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            dmax = fmax(dmax, red[0][k]);
            bmax = fmax(bmax, red[1][k]);
        }
        atomic_max_pos(&out[0], dmax);
        atomic_max_pos(&out[1], bmax);
    }
}

// In-place FFT passes over the grids (plan time, FP64).
struct LdGridX {  // line = row y (grid.y) of grid g (grid.z), positions x
    const double2 *G; int lx, ly, b, ib;
    __device__ double2 operator()(int x, int ch) const {
        const int i = blockIdx.x * ib + ch;
        if (i >= b) return czero<double2>();
        return G[((((int64_t)blockIdx.z * ly + blockIdx.y) * lx) + x) * b + i];
    }
};
struct StGridX {
    double2 *G; int lx, ly, b, ib;
    __device__ void operator()(int x, int ch, double2 v) const {
        const int i = blockIdx.x * ib + ch;
        if (i < b) G[((((int64_t)blockIdx.z * ly + blockIdx.y) * lx) + x) * b + i] = v;
    }
};
struct LdGridY {  // line = column x (grid.y) of grid g, positions y
    const double2 *G; int lx, ly, b, ib;
    __device__ double2 operator()(int y, int ch) const {
        const int i = blockIdx.x * ib + ch;
        if (i >= b) return czero<double2>();
        return G[((((int64_t)blockIdx.z * ly + y) * lx) + blockIdx.y) * b + i];
    }
};
struct StGridY {
    double2 *G; int lx, ly, b, ib;
    __device__ void operator()(int y, int ch, double2 v) const {
        const int i = blockIdx.x * ib + ch;
        if (i < b) G[((((int64_t)blockIdx.z * ly + y) * lx) + blockIdx.y) * b + i] = v;
    }
};

template <typename C> __device__ __forceinline__ C conj_c(C a) {
    a.y = -a.y;
    return a;
}

// U[r][(side*k+s)][kk] = sum_{c < len} x_E[r][edge(side, c, s)] w^(kk c), kk < L of the side.
// One warp per (side*k+s, r, kk).
template <typename R>
__global__ void __launch_bounds__(256) k_side_uhat(const cplx_t<R> *__restrict__ x, cplx_t<R> *__restrict__ U,
                                                   SideMap sm, int64_t N, int64_t NT, int lx, int ly, int lmax,
                                                   int nrhs, const cplx_t<R> *__restrict__ twx,
                                                   const cplx_t<R> *__restrict__ twy) {
    using C = cplx_t<R>;
    const int lane = threadIdx.x & 31;
    const int kk = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int gs = blockIdx.y, r = blockIdx.z;
    const int sg = gs / sm.k, s = gs - sg * sm.k;
    const int L = (sg & 1) ? ly : lx;
    if (kk >= L) return;
    const C *tw = (sg & 1) ? twy : twx;
    const C *xe = x + (int64_t)r * N + NT;
    C acc = czero<C>();
    for (int c = lane; c < sm.len(sg); c += 32) acc = cfma(xe[sm.edge(sg, c, s)], tw[(int)(((int64_t)kk * c) % L)], acc);
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) U[((int64_t)r * 4 * sm.k + gs) * lmax + kk] = acc;
}

// Dot products of one lane chunk, reduced over its 32 lanes by halving
// exchanges: slot j of lane L holds the term of value j ^ (L / (32 / NV)), so
// at every step a lane keeps the low half of its slots and adds the partner's
// high half (no selects); after log2(NV) steps slot 0 holds the partial sum of
// value L / (32 / NV) over the lanes that differ in the top bits, and the
// remaining steps add over the low bits.  The order is fixed by the lane
// numbers, the same for every RHS and every batch.
template <int NV, typename C>
__device__ __forceinline__ C dot_scatter(const C (&g)[NV], C x) {
    C d[NV / 2];
#pragma unroll
    for (int j = 0; j < NV / 2; ++j) {
        const C hi = cmul(g[j + NV / 2], x);
        d[j] = cmul(g[j], x);
        d[j].x += __shfl_xor_sync(0xffffffffu, hi.x, 16);
        d[j].y += __shfl_xor_sync(0xffffffffu, hi.y, 16);
    }
#pragma unroll
    for (int h = NV / 4, m = 8; h >= 1; h >>= 1, m >>= 1)
#pragma unroll
        for (int j = 0; j < h; ++j) {
            d[j].x += __shfl_xor_sync(0xffffffffu, d[j + h].x, m);
            d[j].y += __shfl_xor_sync(0xffffffffu, d[j + h].y, m);
        }
#pragma unroll
    for (int m = 16 / NV; m >= 1; m >>= 1) {
        d[0].x += __shfl_xor_sync(0xffffffffu, d[0].x, m);
        d[0].y += __shfl_xor_sync(0xffffffffu, d[0].y, m);
    }
    return d[0];
}

// Both side products in one pass over the generator spectra, after the block
// product (Y^ holds T^ X^, X^ is intact).  For every frequency f' = (ky, kx),
// lane i and RHS r:
//   Y^[f'][r][i] += sum_gs G^[gs][fa][i] U[r][gs][ka]              (B^T x_E)
//   D[gs][r]      = sum_i G^[gs][fa][i] X^[-f'][r][i]               (B x_T)
// with fa = (ky, -kx), ka = kx on the bottom/top sides and fa = (-ky, kx),
// ka = ky on the right/left sides; D is the term of F_gs(kd), kd = -kx
// (bottom/top) or -ky (right/left).  f' -> fa is one-to-one for every grid,
// so each G^ value is read once and used for both products.
//
// CTA: cx columns x nc chunks of 32 lanes (one warp each) walking ry rows.
// The bottom/top terms of a warp add up over its rows in shared-memory slots
// owned by single lanes; the right/left terms of a row are added over the
// CTA's warps in shared memory.
// Partials P[blk][gs][r][kd] (blk = row block for bottom/top, column block
// for right/left) are summed by k_side_finish in block order.  Every order
// depends on the geometry only (b, lx, ly, the SM count), not on the batch.
// Per-thread asynchronous copy of one element (8 or 16 bytes) into shared
// memory, zero-filled when !ok (no bytes read); completion is waited per
// thread (cp.async groups), so a thread may read back only its own copies.
template <typename C> __device__ __forceinline__ void cp_async_elem(C *dst, const C *src, bool ok) {
    const uint32_t d = smem_u32(dst);
    const int n = ok ? (int)sizeof(C) : 0;
    if constexpr (sizeof(C) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bit j of the result is bit j ^ p of m (NV bits): adjacent blocks of width
// 2^s swapped for every set bit s of p.
template <int NV> __device__ __forceinline__ uint32_t xor_permute_bits(uint32_t m, int p) {
    constexpr uint32_t M[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
    for (int sh = 0; (1 << sh) < NV; ++sh)
        if ((p >> sh) & 1) m = ((m & M[sh]) << (1 << sh)) | ((m >> (1 << sh)) & M[sh]);
    return m;
}

template <typename R, int NV, int RB>
__global__ void __launch_bounds__(256, 2) k_side_fused(const cplx_t<R> *__restrict__ Gh,
                                                    const cplx_t<R> *__restrict__ Xh, cplx_t<R> *__restrict__ Yh,
                                                    const cplx_t<R> *__restrict__ U, cplx_t<R> *__restrict__ P,
                                                    int ng, uint32_t btmask, int b, int lx, int ly, int lmax,
                                                    int nrhs, int nc, int cx, int ry) {
    using C = cplx_t<R>;
    constexpr int RQ = side_rq<R>(NV), GSZ = 32 / NV;
    static_assert(RB % RQ == 0, "RHS block must be a multiple of RQ");
    extern __shared__ __align__(16) unsigned char zt_smem[];
    const int W = (int)(blockDim.x >> 5), nsl = cx + ry;
    C *su = reinterpret_cast<C *>(zt_smem);  // [nsl][RB][NV] U at the CTA's columns, then rows
    C *srl = su + nsl * NV * RB;             // [ry][W][RB][NV] right/left terms per row and warp
    C *sbt = srl + ry * W * RB * NV;         // [W][RB][NV] bottom/top sums of each warp
    C *sg = sbt + W * RB * NV;               // [2][NV][threads] G^ of the current and the next row (FP32)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nthr = (int)blockDim.x;
    const int ic = wid % nc, cxl = wid / nc;
    const int x0 = blockIdx.x * cx, y0 = blockIdx.y * ry;
    const int kx = x0 + cxl, nkx = kx == 0 ? 0 : lx - kx;
    const int i = ic * 32 + lane;
    const bool iok = kx < lx && i < b;
    const int nrow = min(ry, ly - y0);
    const int perm = lane / GSZ;
    // slot j holds value j ^ perm: is it a grid, a bottom/top grid
    const uint32_t real = xor_permute_bits<NV>(ng >= 32 ? 0xffffffffu : (1u << ng) - 1u, perm);
    const uint32_t btm = xor_permute_bits<NV>(btmask, perm);
    const bool v0bt = (btmask >> perm) & 1, leader = lane % GSZ == 0;
    const int F = lx * ly;
    const int sv = threadIdx.x % NV, sstep = nthr / NV;  // staging and sums: value per thread
    // G^ of row yl (bottom/top at (ky, -kx), right/left at (-ky, kx)) into stage st
    auto issue_row = [&](int yl, int st) {
        const int ky = y0 + yl, nky = ky == 0 ? 0 : ly - ky;
        const int fbt = ky * lx + nkx, frl = nky * lx + kx;
        C *dst = sg + st * NV * nthr + threadIdx.x;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const bool ok = iok && ((real >> j) & 1);
            const C *src = ok ? Gh + ((j ^ perm) * F + ((btm >> j) & 1 ? fbt : frl)) * b + i : Gh;
            cp_async_elem(dst + j * nthr, src, ok);
        }
        cp_async_commit();
    };
    for (int rb0 = 0; rb0 < nrhs; rb0 += RB) {
        const int rbn = min(RB, nrhs - rb0);
        __syncthreads();  // shared memory of the previous RHS block consumed
        if (side_prefetch<R>()) issue_row(0, 0);
        for (int e = threadIdx.x / NV; e < nsl * rbn; e += sstep) {
            const int sl = e / rbn, q = e - sl * rbn;
            const bool bt = (btmask >> sv) & 1;
            const int kk = sl < cx ? x0 + sl : y0 + sl - cx;
            const bool ok = sv < ng && (sl < cx ? bt && kk < lx : !bt && kk < ly);
            su[(sl * RB + q) * NV + sv] = ok ? U[((int64_t)(rb0 + q) * ng + sv) * lmax + kk] : czero<C>();
        }
        __syncthreads();
        // bottom/top sums of this warp: one slot per (RHS, value), owned by the
        // lane that holds the value after the reduction
        C *acc = sbt + wid * RB * NV + perm;
        if (leader && v0bt)
            for (int q = 0; q < rbn; ++q) acc[q * NV] = czero<C>();
        for (int yl = 0; yl < nrow; ++yl) {  // no barrier inside: the warps walk their columns independently
            const int ky = y0 + yl, nky = ky == 0 ? 0 : ly - ky;
            C g[NV];
            if constexpr (side_prefetch<R>()) {
                if (yl + 1 < nrow) {  // the next row's copies in flight while this row is computed
                    issue_row(yl + 1, (yl + 1) & 1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                const C *gs = sg + (yl & 1) * NV * nthr + threadIdx.x;
#pragma unroll
                for (int j = 0; j < NV; ++j) g[j] = gs[j * nthr];
            } else {
                const int fbt = ky * lx + nkx, frl = nky * lx + kx;
#pragma unroll
                for (int j = 0; j < NV; ++j)
                    g[j] = iok && ((real >> j) & 1) ? Gh[((j ^ perm) * F + ((btm >> j) & 1 ? fbt : frl)) * b + i]
                                                   : czero<C>();
            }
            int uoff[NV];  // U of slot j: su + uoff[j] + q NV
#pragma unroll
            for (int j = 0; j < NV; ++j) uoff[j] = ((btm >> j) & 1 ? cxl : cx + yl) * RB * NV + (j ^ perm);
            const int64_t fneg = (int64_t)nky * lx + nkx, fpos = (int64_t)ky * lx + kx;
            C *rowl = srl + (yl * W + wid) * RB * NV + perm;
#pragma unroll 1
            for (int q0 = 0; q0 < rbn; q0 += RQ) {
                C xv[RQ], yv[RQ];
#pragma unroll
                for (int q = 0; q < RQ; ++q) {
                    const bool ok = iok && q0 + q < rbn;
                    const int64_t r = rb0 + q0 + q;
                    xv[q] = ok ? Xh[(fneg * nrhs + r) * b + i] : czero<C>();
                    yv[q] = ok ? Yh[(fpos * nrhs + r) * b + i] : czero<C>();
                }
                const C *uq = su + q0 * NV;
#pragma unroll
                for (int q = 0; q < RQ; ++q) {
                    if (q0 + q >= rbn) break;  // uniform over the CTA
#pragma unroll
                    for (int j = 0; j < NV; ++j) yv[q] = cfma(g[j], uq[uoff[j] + q * NV], yv[q]);
                    const C dq = dot_scatter<NV>(g, xv[q]);
                    if (leader) {
                        if (v0bt) acc[(q0 + q) * NV] = acc[(q0 + q) * NV] + dq;
                        rowl[(q0 + q) * NV] = dq;
                    }
                    if (iok) Yh[(fpos * nrhs + rb0 + q0 + q) * b + i] = yv[q];
                }
            }
        }
        __syncthreads();
        if (sv < ng) {
            if ((btmask >> sv) & 1) {  // bottom/top: over the lane chunks of each column in order
                for (int e = threadIdx.x / NV; e < cx * rbn; e += sstep) {
                    const int c = e / rbn, q = e - c * rbn;
                    const int col = x0 + c;
                    if (col < lx) {
                        C s2 = sbt[((c * nc) * RB + q) * NV + sv];
                        for (int h = 1; h < nc; ++h) s2 = s2 + sbt[((c * nc + h) * RB + q) * NV + sv];
                        P[(((int64_t)blockIdx.y * ng + sv) * nrhs + rb0 + q) * lmax + (col == 0 ? 0 : lx - col)] = s2;
                    }
                }
            } else {  // right/left: over the CTA's warps in order, per row
                for (int e = threadIdx.x / NV; e < nrow * rbn; e += sstep) {
                    const int yl = e / rbn, q = e - yl * rbn;
                    const int ky = y0 + yl, nky = ky == 0 ? 0 : ly - ky;
                    const C *pr = srl + (yl * W) * RB * NV + q * NV + sv;
                    C t = pr[0];
                    for (int w = 1; w < W; ++w) t = t + pr[w * RB * NV];
                    P[(((int64_t)blockIdx.x * ng + sv) * nrhs + rb0 + q) * lmax + nky] = t;
                }
            }
        }
    }
}

// y_E[r][e] = 1/(Lx Ly) sum_kk w^(-c kk) F_gs[r][kk] + sum_j C[e][j] x_E[r][j],
// F_gs the sum of the fused kernel's partials (blocks in four interleaved
// parts, each in block order, then the parts in order: fixed by the geometry).
// CTA per (grid gs, RHS, 8 cells of the side): the sums once into shared
// memory, then one warp per edge unknown with fixed-order warp sums.
template <typename R>
__global__ void __launch_bounds__(256) k_side_finish(const cplx_t<R> *__restrict__ x, const cplx_t<R> *__restrict__ Cm,
                                                     const cplx_t<R> *__restrict__ P, cplx_t<R> *__restrict__ y,
                                                     SideMap sm, int64_t N, int64_t NT, int E, int lx, int ly,
                                                     int lmax, int nrhs, int nblk_bt, int nblk_rl,
                                                     const cplx_t<R> *__restrict__ twx,
                                                     const cplx_t<R> *__restrict__ twy) {
    using C = cplx_t<R>;
    extern __shared__ __align__(16) unsigned char zt_smem[];
    C *fs = reinterpret_cast<C *>(zt_smem);  // [L]
    const int gs = blockIdx.x, r = blockIdx.y;
    const int k = sm.k, ng = 4 * k;
    const int sg = gs / k, s = gs - sg * k;
    const int len = sm.len(sg);
    const int c0 = blockIdx.z * 8;
    if (c0 >= len) return;  // uniform over the CTA
    const int L = (sg & 1) ? ly : lx;
    const int nblk = (sg & 1) ? nblk_rl : nblk_bt;
    // thread (kk, part): blocks part, part + 4, ... (loads issued together),
    // then the four parts' sums added in block order through shared memory
    constexpr int NP = 4, BU = 8;
    C *part = fs + lmax;  // [NP][L]
    const int64_t bstride = (int64_t)ng * nrhs * lmax;
    for (int t = threadIdx.x; t < NP * L; t += blockDim.x) {
        const int kk = t % L, pt = t / L;
        const C *pp = P + ((int64_t)gs * nrhs + r) * lmax + kk;
        C acc = czero<C>();
        for (int b0 = pt; b0 < nblk; b0 += NP * BU) {
            C v[BU];
#pragma unroll
            for (int u = 0; u < BU; ++u) {
                const int blk = b0 + u * NP;
                v[u] = blk < nblk ? pp[blk * bstride] : czero<C>();
            }
#pragma unroll
            for (int u = 0; u < BU; ++u) acc = acc + v[u];
        }
        part[pt * L + kk] = acc;
    }
    __syncthreads();
    for (int kk = threadIdx.x; kk < L; kk += blockDim.x) {
        C t = part[kk];
#pragma unroll
        for (int pt = 1; pt < NP; ++pt) t = t + part[pt * L + kk];
        fs[kk] = t;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int c = c0 + (threadIdx.x >> 5);
    if (c >= len) return;
    const int e = sm.edge(sg, c, s);
    const C *tw = (sg & 1) ? twy : twx;
    C a = czero<C>();
    for (int kk = lane; kk < L; kk += 32) a = cfma(conj_c(tw[(c * kk) % L]), fs[kk], a);
    const C *crow = Cm + (int64_t)e * E;
    const C *xe = x + (int64_t)r * N + NT;
    C b2 = czero<C>();
    for (int j = lane; j < E; j += 32) b2 = cfma(crow[j], xe[j], b2);
    for (int o = 16; o > 0; o >>= 1) {
        a.x += __shfl_xor_sync(0xffffffffu, a.x, o);
        a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
        b2.x += __shfl_xor_sync(0xffffffffu, b2.x, o);
        b2.y += __shfl_xor_sync(0xffffffffu, b2.y, o);
    }
    if (lane == 0) {
        const R sc = (R)(1.0 / ((double)lx * (double)ly));
        y[(int64_t)r * N + NT + e] = cscale(a, sc) + b2;
    }
}

unsigned grid1d(int64_t n, int threads, int nsm) {
    const int64_t g = (n + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)nsm * 16));
}

}  // namespace

// Plan time: generator grids from B, structure check, 2-D spectra (FP64 and FP32).
ztoep_status_t sides_build(ztoep_plan_t p, const double2 *B, cudaStream_t s, size_t *acc) {
    const SideMap sm{p->nx, p->ny, p->side_k};
    const int b = p->b, lx = p->lx, ly = p->ly;
    const int ng = 4 * sm.k;
    const size_t count = (size_t)ng * p->F * b;
    ZT_TRY(dalloc((void **)&p->G64, sizeof(double2) * count, acc));
    ZT_TRY(dalloc((void **)&p->G32, sizeof(float2) * count, acc));
    {
        KScope ks(K_MISC, s);
        k_side_embed<<<grid1d((int64_t)count, 256, p->nsm), 256, 0, s>>>(B, p->G64, sm, b, lx, ly, p->NT);
        ZT_CUDA(cudaGetLastError());
    }
    unsigned long long *dev = nullptr;
    ZT_TRY(dalloc((void **)&dev, 2 * sizeof(unsigned long long), nullptr));
    ztoep_status_t st = ZTOEP_OK;
    unsigned long long host[2] = {0, 0};
    if (cudaMemsetAsync(dev, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) st = ZTOEP_ERR_CUDA;
    if (st == ZTOEP_OK) {
        KScope ks(K_MISC, s);
        k_side_verify<<<grid1d((int64_t)p->E * p->NT, 256, p->nsm), 256, 0, s>>>(B, p->G64, sm, b, lx, ly, p->NT,
                                                                                 p->E, dev);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(host, dev, sizeof host, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            st = ZTOEP_ERR_CUDA;
    }
    cudaFree(dev);
    ZT_TRY(st);
    double dmax, bmax;
    std::memcpy(&dmax, &host[0], sizeof dmax);
    std::memcpy(&bmax, &host[1], sizeof bmax);
    if (!(dmax <= 1e-11 * bmax)) return ZTOEP_ERR_ARG;  // B does not have the declared layout (or is not finite)
    // 2-D FFT of every grid, in place: along x (lines = rows), then along y (lines = columns)
    const int libx = pick_lib(lx, b, sizeof(double2), 64 * 1024, 32);
    const int ibx = 1 << libx;
    dim3 gx((b + ibx - 1) / ibx, ly, ng);
    ZT_TRY((launch_fft_pass<double>(p->fx, p->twx64, libx, false, gx, LdGridX{p->G64, lx, ly, b, ibx},
                                    StGridX{p->G64, lx, ly, b, ibx}, s)));
    const int liby = pick_lib(ly, b, sizeof(double2), 64 * 1024, 32);
    const int iby = 1 << liby;
    dim3 gy((b + iby - 1) / iby, lx, ng);
    ZT_TRY((launch_fft_pass<double>(p->fy, p->twy64, liby, false, gy, LdGridY{p->G64, lx, ly, b, iby},
                                    StGridY{p->G64, lx, ly, b, iby}, s)));
    return launch_c128_to_c64(p->G64, p->G32, (int64_t)count, s);
}

template <typename R> static const cplx_t<R> *gh_of(ztoep_plan_t p);
template <> const float2 *gh_of<float>(ztoep_plan_t p) { return p->G32; }
template <> const double2 *gh_of<double>(ztoep_plan_t p) { return p->G64; }
template <typename R> static const cplx_t<R> *tw_x(ztoep_plan_t p);
template <> const float2 *tw_x<float>(ztoep_plan_t p) { return p->twx32; }
template <> const double2 *tw_x<double>(ztoep_plan_t p) { return p->twx64; }
template <typename R> static const cplx_t<R> *tw_y(ztoep_plan_t p);
template <> const float2 *tw_y<float>(ztoep_plan_t p) { return p->twy32; }
template <> const double2 *tw_y<double>(ztoep_plan_t p) { return p->twy64; }
template <typename R> static const cplx_t<R> *cm_of(ztoep_plan_t p);
template <> const float2 *cm_of<float>(ztoep_plan_t p) { return p->C32; }
template <> const double2 *cm_of<double>(ztoep_plan_t p) { return p->C64; }

// Side slices of x_E to the frequency domain.
template <typename R>
ztoep_status_t sides_uhat(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, MatvecWs &w, cudaStream_t s) {
    const SideMap sm{p->nx, p->ny, p->side_k};
    const int lmax = std::max(p->lx, p->ly);
    KScope ks(K_EDGE, s);
    k_side_uhat<R><<<dim3((lmax + 7) / 8, 4 * sm.k, nrhs), 256, 0, s>>>(
        x, reinterpret_cast<cplx_t<R> *>(w.Us), sm, p->N, p->NT, p->lx, p->ly, lmax, nrhs, tw_x<R>(p), tw_y<R>(p));
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

namespace {

// Launch geometry of k_side_fused: nc chunks of 32 lanes cover b, cx columns
// per CTA (about 8 warps), ry rows per CTA (about three CTAs per SM over the
// grid, shared memory within the default 48 KB).
struct SideGeom {
    int nc, cx, ry, nxb, nyb;
};

int side_nv(int k) { return 4 * k <= 4 ? 4 : 4 * k <= 8 ? 8 : 4 * k <= 16 ? 16 : 32; }

// Shared memory of k_side_fused: U, the per-row and per-warp sums (these grow
// with ry), and two stages of G^ rows (one element per thread and grid).
template <typename R> size_t side_smem_sums(int nv, int cx, int nc, int ry) {
    const int rb = side_rb<R>(), warps = cx * nc;
    return sizeof(cplx_t<R>) * ((size_t)rb * (cx + ry) * nv + (size_t)ry * warps * rb * nv + (size_t)warps * rb * nv);
}
template <typename R> size_t side_smem(int nv, int cx, int nc, int ry) {
    return side_smem_sums<R>(nv, cx, nc, ry) + (side_prefetch<R>() ? sizeof(cplx_t<R>) * 2 * nv * 32 * cx * nc : 0);
}

SideGeom side_geom(ztoep_plan_t p) {
    SideGeom g;
    g.nc = (p->b + 31) / 32;
    g.cx = std::max(1, 8 / g.nc);
    g.nxb = (p->lx + g.cx - 1) / g.cx;
    const int nv = side_nv(p->side_k);
    g.ry = std::max(1, std::min({32, p->ly, g.nxb * p->ly / (3 * std::max(p->nsm, 1))}));
    while (g.ry > 1 &&
           std::max(side_smem_sums<float>(nv, g.cx, g.nc, g.ry), side_smem_sums<double>(nv, g.cx, g.nc, g.ry)) >
               48 * 1024)
        --g.ry;
    g.nyb = (p->ly + g.ry - 1) / g.ry;
    return g;
}

}  // namespace

int64_t sides_partials(ztoep_plan_t p) {
    const SideGeom g = side_geom(p);
    return (int64_t)std::max(g.nxb, g.nyb) * 4 * p->side_k * std::max(p->lx, p->ly);
}

// Both side products in one pass (after the block product): Y^ += B^T x_E
// terms, and the partials of B x_T.
template <typename R>
ztoep_status_t sides_fused(ztoep_plan_t p, int nrhs, const cplx_t<R> *Xh, cplx_t<R> *Yh, MatvecWs &w,
                           cudaStream_t s) {
    const SideMap sm{p->nx, p->ny, p->side_k};
    const int lmax = std::max(p->lx, p->ly);
    const SideGeom g = side_geom(p);
    const int nv = side_nv(sm.k), threads = 32 * g.cx * g.nc, ng = 4 * sm.k;
    uint32_t btmask = 0;  // grids of the bottom (side 0) and top (side 2) sides
    for (int v = 0; v < ng; ++v)
        if (((v / sm.k) & 1) == 0) btmask |= 1u << v;
    const size_t smem = side_smem<R>(nv, g.cx, g.nc, g.ry);
    const dim3 grid(g.nxb, g.nyb);
    const cplx_t<R> *U = reinterpret_cast<const cplx_t<R> *>(w.Us);
    cplx_t<R> *P = reinterpret_cast<cplx_t<R> *>(w.Ps);
    constexpr int RB = side_rb<R>();
    KScope ks(K_EDGE, s);
#define ZT_FUSED(NV)                                                                                              \
    {                                                                                                             \
        static bool attr = false;                                                                                 \
        if (!attr) {                                                                                              \
            ZT_CUDA(cudaFuncSetAttribute(k_side_fused<R, NV, RB>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                         227 * 1024));                                                            \
            attr = true;                                                                                          \
        }                                                                                                         \
        k_side_fused<R, NV, RB><<<grid, threads, smem, s>>>(gh_of<R>(p), Xh, Yh, U, P, ng, btmask, p->b, p->lx,   \
                                                            p->ly, lmax, nrhs, g.nc, g.cx, g.ry);                 \
    }
    switch (nv) {
        case 4: ZT_FUSED(4); break;
        case 8: ZT_FUSED(8); break;
        case 16: ZT_FUSED(16); break;
        default: ZT_FUSED(32); break;
    }
#undef ZT_FUSED
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// y_E = B x_T + C x_E from the fused kernel's partials.
template <typename R>
ztoep_status_t sides_finish(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *y, MatvecWs &w,
                            cudaStream_t s) {
    const SideMap sm{p->nx, p->ny, p->side_k};
    const int lmax = std::max(p->lx, p->ly);
    const SideGeom g = side_geom(p);
    const dim3 grid(4 * sm.k, nrhs, (std::max(p->nx, p->ny) + 7) / 8);
    KScope ks(K_EDGE, s);
    k_side_finish<R><<<grid, 256, sizeof(cplx_t<R>) * 5 * lmax, s>>>(
        x, cm_of<R>(p), reinterpret_cast<const cplx_t<R> *>(w.Ps), y, sm, p->N, p->NT, p->E, p->lx, p->ly, lmax,
        nrhs, g.nyb, g.nxb, tw_x<R>(p), tw_y<R>(p));
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

#define ZT_SIDES_INST(R)                                                                                       \
    template ztoep_status_t sides_uhat<R>(ztoep_plan_t, int, const cplx_t<R> *, MatvecWs &, cudaStream_t);        \
    template ztoep_status_t sides_fused<R>(ztoep_plan_t, int, const cplx_t<R> *, cplx_t<R> *, MatvecWs &,          \
                                           cudaStream_t);                                                          \
    template ztoep_status_t sides_finish<R>(ztoep_plan_t, int, const cplx_t<R> *, cplx_t<R> *, MatvecWs &,         \
                                            cudaStream_t);
ZT_SIDES_INST(float)
ZT_SIDES_INST(double)

}  // namespace ztoep
