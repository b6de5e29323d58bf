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

// Fs[(side*k+s)][r][kk] = sum_{cross, i} G^[..][f][i] X^[flip][r][i].  One
// CTA per (axis, kk, chunk of RQ RHS) serves both sides of the axis (bottom
// and top share the column kx of X^, right and left the row ky), so X^ is
// read twice in all.  Each thread walks a fixed strided subset of the
// K = L_cross * b pairs, two at a time (one for k > 4) with every load issued first, and keeps
// 2 x KS x RQ sums in registers; the CTA adds the per-thread sums by a warp tree
// and the 8 warp sums in order.  The order depends on K and blockDim only, so a
// RHS is summed identically alone and in any batch.
template <typename R, int KS, int RQ>
__global__ void __launch_bounds__(256) k_side_dot(const cplx_t<R> *__restrict__ Gh, const cplx_t<R> *__restrict__ Xh,
                                                  cplx_t<R> *__restrict__ Fs, SideMap sm, int b, int lx, int ly,
                                                  int lmax, int nrhs) {
    using C = cplx_t<R>;
    constexpr int NO = 2 * KS * RQ, U = KS > 4 ? 1 : 2;
    __shared__ C red[8][NO];
    const int ax = blockIdx.y < lx ? 0 : 1;  // 0: kk = kx (sides 0, 2); 1: kk = ky (sides 1, 3)
    const int kk = ax == 0 ? blockIdx.y : blockIdx.y - lx;
    const int k = sm.k;
    const int r0 = blockIdx.x * RQ;
    const int rc = min(RQ, nrhs - r0);
    const int lcross = ax ? lx : ly;
    const int K = lcross * b;
    const int64_t F = (int64_t)lx * ly;
    const int64_t gstride = F * b;
    const C *g0 = Gh + (int64_t)ax * k * gstride;        // side ax
    const C *g1 = Gh + (int64_t)(ax + 2) * k * gstride;  // side ax + 2
    C acc[2][KS][RQ];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int s = 0; s < KS; ++s)
#pragma unroll
            for (int q = 0; q < RQ; ++q) acc[h][s][q] = czero<C>();
    for (int kb = threadIdx.x; kb < K; kb += U * blockDim.x) {
        C xv[U][RQ], gv[U][2][KS];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int kg = kb + u * blockDim.x;
            const bool ok = kg < K;
            const int cross = ok ? kg / b : 0, i = ok ? kg - cross * b : 0;
            const int64_t f = ax ? (int64_t)kk * lx + cross : (int64_t)cross * lx + kk;
            const int64_t fl = ax ? (int64_t)kk * lx + (lx - cross) % lx : (int64_t)((ly - cross) % ly) * lx + kk;
#pragma unroll
            for (int q = 0; q < RQ; ++q) xv[u][q] = (ok && q < rc) ? Xh[(fl * nrhs + r0 + q) * b + i] : czero<C>();
#pragma unroll
            for (int s = 0; s < KS; ++s) {
                const bool sk = ok && s < k;
                gv[u][0][s] = sk ? g0[(int64_t)s * gstride + f * b + i] : czero<C>();
                gv[u][1][s] = sk ? g1[(int64_t)s * gstride + f * b + i] : czero<C>();
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int s = 0; s < KS; ++s)
#pragma unroll
                    for (int q = 0; q < RQ; ++q) acc[h][s][q] = cfma(gv[u][h][s], xv[u][q], acc[h][s][q]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int s = 0; s < KS; ++s)
#pragma unroll
            for (int q = 0; q < RQ; ++q) {
                C v = acc[h][s][q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
                }
                if (lane == 0) red[w][(h * KS + s) * RQ + q] = v;
            }
    __syncthreads();
    for (int o = threadIdx.x; o < NO; o += blockDim.x) {
        const int h = o / (KS * RQ), s = (o / RQ) % KS, q = o % RQ;
        if (s < k && q < rc) {
            C t = red[0][o];
            for (int ww = 1; ww < (int)(blockDim.x >> 5); ++ww) t = t + red[ww][o];
            Fs[((int64_t)((ax + 2 * h) * k + s) * nrhs + r0 + q) * lmax + kk] = t;
        }
    }
}

// y_E[r][e] = 1/(Lx Ly) sum_kk w^(-c kk) Fs[(side*k+s)][r][kk] + sum_j C[e][j] x_E[r][j].
// One warp per (e, r); fixed-order warp sums.
template <typename R>
__global__ void __launch_bounds__(256) k_side_finish(const cplx_t<R> *__restrict__ x, const cplx_t<R> *__restrict__ Cm,
                                                     const cplx_t<R> *__restrict__ Fs, cplx_t<R> *__restrict__ y,
                                                     SideMap sm, int64_t N, int64_t NT, int E, int lx, int ly,
                                                     int lmax, int nrhs, const cplx_t<R> *__restrict__ twx,
                                                     const cplx_t<R> *__restrict__ twy) {
    using C = cplx_t<R>;
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * 8 + (threadIdx.x >> 5), r = blockIdx.y;
    if (e >= E) return;
    int sg, c, s;
    sm.locate(e, sg, c, s);
    const int L = (sg & 1) ? ly : lx;
    const C *tw = (sg & 1) ? twy : twx;
    const C *fs = Fs + ((int64_t)(sg * sm.k + s) * nrhs + r) * lmax;
    C a = czero<C>();
    for (int kk = lane; kk < L; kk += 32) a = cfma(conj_c(tw[(int)(((int64_t)c * kk) % L)]), fs[kk], a);
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

// Y^[f][r][i] += sum_{side,s} G^[side,s][flip][i] U[r][side,s][kk]: thread per
// (f, i); the thread's 4k spectrum values (in chunks of GC) and the offsets of
// the matching U entries are loaded once and applied to every RHS; the terms
// are added in (side, s) order whatever GC is (a chunk boundary is a store and
// reload of the running sum, exact in its precision).
template <typename R, int GC>
__global__ void __launch_bounds__(256) k_side_add(const cplx_t<R> *__restrict__ Gh, const cplx_t<R> *__restrict__ U,
                                                  cplx_t<R> *__restrict__ Yh, SideMap sm, int b, int lx, int ly,
                                                  int lmax, int nrhs) {
    using C = cplx_t<R>;
    const int64_t F = (int64_t)lx * ly;
    const int64_t total = F * b;
    const int ng = 4 * sm.k;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = idx / b;
        const int i = (int)(idx - f * b);
        const int ky = (int)(f / lx), kx = (int)(f - (int64_t)ky * lx);
        const int64_t fx = (int64_t)ky * lx + (lx - kx) % lx;    // bottom / top: G^[ky][-kx]
        const int64_t fy = (int64_t)((ly - ky) % ly) * lx + kx;  // right / left: G^[-ky][kx]
        for (int g0 = 0; g0 < ng; g0 += GC) {
            const int gn = min(GC, ng - g0);
            C gv[GC];
            int uo[GC];
#pragma unroll
            for (int j = 0; j < GC; ++j) {
                const int gs = g0 + (j < gn ? j : 0);
                const bool odd = (gs / sm.k) & 1;
                gv[j] = j < gn ? Gh[((int64_t)gs * F + (odd ? fy : fx)) * b + i] : czero<C>();
                uo[j] = gs * lmax + (odd ? ky : kx);
            }
            const C *ur = U;
            for (int r = 0; r < nrhs; ++r, ur += (int64_t)ng * lmax) {
                C acc = Yh[(f * nrhs + r) * b + i];
#pragma unroll
                for (int j = 0; j < GC; ++j)
                    if (j < gn) acc = cfma(gv[j], ur[uo[j]], acc);
                Yh[(f * nrhs + r) * b + i] = acc;
            }
        }
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

// B x_T per side in the frequency domain (reads X^), then y_E = B x_T + C x_E.
template <typename R>
ztoep_status_t sides_edge_rows(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, const cplx_t<R> *Xh, cplx_t<R> *y,
                               MatvecWs &w, cudaStream_t s) {
    const SideMap sm{p->nx, p->ny, p->side_k};
    const int lmax = std::max(p->lx, p->ly);
    cplx_t<R> *Fs = reinterpret_cast<cplx_t<R> *>(w.Fs);
    KScope ks(K_EDGE, s);
    ks.add(1);
    // RHS per CTA: 2 for FP32 with k <= 4, else 1 (registers); RHS chunks of a line are adjacent (G^ from L2)
    constexpr bool F32 = sizeof(R) == sizeof(float);
    if (sm.k <= 4) {
        constexpr int RQ = F32 ? 2 : 1;
        dim3 gd((nrhs + RQ - 1) / RQ, p->lx + p->ly);
        k_side_dot<R, 4, RQ><<<gd, 256, 0, s>>>(gh_of<R>(p), Xh, Fs, sm, p->b, p->lx, p->ly, lmax, nrhs);
    } else {
        dim3 gd(nrhs, p->lx + p->ly);
        k_side_dot<R, 8, 1><<<gd, 256, 0, s>>>(gh_of<R>(p), Xh, Fs, sm, p->b, p->lx, p->ly, lmax, nrhs);
    }
    k_side_finish<R><<<dim3((p->E + 7) / 8, nrhs), 256, 0, s>>>(x, cm_of<R>(p), Fs, y, sm, p->N, p->NT, p->E, p->lx,
                                                                 p->ly, lmax, nrhs, tw_x<R>(p), tw_y<R>(p));
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

// B^T x_E terms added to Y^ (after the block product).
template <typename R>
ztoep_status_t sides_add(ztoep_plan_t p, int nrhs, cplx_t<R> *Yh, MatvecWs &w, cudaStream_t s) {
    const SideMap sm{p->nx, p->ny, p->side_k};
    const int lmax = std::max(p->lx, p->ly);
    KScope ks(K_EDGE, s);
    const unsigned g = grid1d((int64_t)p->F * p->b, 256, p->nsm);
    const cplx_t<R> *U = reinterpret_cast<const cplx_t<R> *>(w.Us);
    if (nrhs >= 8)  // many RHS: one pass over Y^ per 16 terms
        k_side_add<R, 16><<<g, 256, 0, s>>>(gh_of<R>(p), U, Yh, sm, p->b, p->lx, p->ly, lmax, nrhs);
    else  // few RHS: fewer registers, more CTAs resident
        k_side_add<R, 8><<<g, 256, 0, s>>>(gh_of<R>(p), U, Yh, sm, p->b, p->lx, p->ly, lmax, nrhs);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

#define ZT_SIDES_INST(R)                                                                                          \
    template ztoep_status_t sides_uhat<R>(ztoep_plan_t, int, const cplx_t<R> *, MatvecWs &, cudaStream_t);           \
    template ztoep_status_t sides_edge_rows<R>(ztoep_plan_t, int, const cplx_t<R> *, const cplx_t<R> *, cplx_t<R> *, \
                                               MatvecWs &, cudaStream_t);                                             \
    template ztoep_status_t sides_add<R>(ztoep_plan_t, int, cplx_t<R> *, MatvecWs &, cudaStream_t);
ZT_SIDES_INST(float)
ZT_SIDES_INST(double)

}  // namespace ztoep
