// FP64 complex Gauss-Jordan elimination with partial pivoting (gj.cuh).
#include <algorithm>

#include "gj.cuh"
#include "instrument.cuh"

namespace ztoep {
namespace {

__device__ __forceinline__ double2 crecip(double2 z) {
    const double d = z.x * z.x + z.y * z.y;
    return make_double2(z.x / d, -z.y / d);
}

// Step k, one CTA: pivot row = argmax_{i >= k} |W[i][k]| (ties: lowest i),
// swap it into row k (all w2 columns), then prow = W[k][:] / W[k][k] and
// col = W[:][k].  A zero
// or non-finite pivot sets *err.
__global__ void __launch_bounds__(1024) k_gj_pivot(double2 *W, int p, int w2, int k, double2 *col, double2 *prow, int *err) {
    __shared__ double s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_piv;
    double best = -1.0;
    int bi = k;
    for (int i = k + threadIdx.x; i < p; i += blockDim.x) {
        const double2 z = W[(int64_t)i * w2 + k];
        const double m = z.x * z.x + z.y * z.y;
        if (m > best) {  // strict: the lowest index wins ties within a thread
            best = m;
            bi = i;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
            best = ob;
            bi = oi;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_v[warp] = best;
        s_i[warp] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = s_v[0];
        int ib = s_i[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
            if (s_v[q] > bv || (s_v[q] == bv && s_i[q] < ib)) {
                bv = s_v[q];
                ib = s_i[q];
            }
        if (!(bv > 0.0) || !isfinite(bv)) atomicOr(err, 1);
        s_piv = ib;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != k)
        for (int j = threadIdx.x; j < w2; j += blockDim.x) {
            const double2 t = W[(int64_t)k * w2 + j];
            W[(int64_t)k * w2 + j] = W[(int64_t)piv * w2 + j];
            W[(int64_t)piv * w2 + j] = t;
        }
    __syncthreads();
    const double2 inv = crecip(W[(int64_t)k * w2 + k]);
    for (int j = threadIdx.x; j < w2; j += blockDim.x) prow[j] = cmul(W[(int64_t)k * w2 + j], inv);
    for (int i = threadIdx.x; i < p; i += blockDim.x) col[i] = W[(int64_t)i * w2 + k];
}

// Step k, all rows: row k <- prow, row i <- row i - col[i] prow; column k
// becomes exactly the unit vector e_k.
__global__ void k_gj_elim(double2 *W, int p, int w2, int k, const double2 *__restrict__ col,
                          const double2 *__restrict__ prow) {
    const int64_t total = (int64_t)p * w2;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx / w2), j = (int)(idx - (int64_t)i * w2);
        if (j == k) {
            W[idx] = make_double2(i == k ? 1.0 : 0.0, 0.0);
        } else if (i == k) {
            W[idx] = prow[j];
        } else {
            const double2 c = col[i], r = prow[j];
            double2 v = W[idx];
            v.x -= c.x * r.x - c.y * r.y;
            v.y -= c.x * r.y + c.y * r.x;
            W[idx] = v;
        }
    }
}

}  // namespace

ztoep_status_t gj_solve(double2 *W, int p, int w, double2 *col, double2 *prow, int *err, cudaStream_t s) {
    const int pt = std::min(1024, std::max(32, (p + 31) / 32 * 32));
    const unsigned ge = (unsigned)std::min<int64_t>(((int64_t)p * w + 255) / 256, 4096);
    for (int k = 0; k < p; ++k) {
        KScope ks(K_MISC, s);
        ks.add(2);
        k_gj_pivot<<<1, pt, 0, s>>>(W, p, w, k, col, prow, err);
        k_gj_elim<<<ge, 256, 0, s>>>(W, p, w, k, col, prow);
        ZT_CUDA(cudaGetLastError());
    }
    return ZTOEP_OK;
}

}  // namespace ztoep
