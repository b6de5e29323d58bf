// Port matrices after a delta-port solve (Sec. IV-B): the port currents
// I^[a][k] = I[k][i_a], the admittance Y = L I^ L (L = diag(1 / l_{i_k})) and
// the power-wave scattering matrix with real reference impedances z0,
//   S = F (Z_port - G)(Z_port + G)^-1 F^-1,  Z_port = Y^-1,
//   G = diag(z0), F = diag(1 / (2 sqrt(z0))).
// With Z_port = Y^-1, (Z_port - G)(Z_port + G)^-1 = (I - G Y)(I + G Y)^-1,
// so no inverse of Y is formed: S'^T solves (I + G Y)^T S'^T = (I - G Y)^T,
// by Gauss-Jordan elimination with partial pivoting on the p x 2p array
// [ (I + G Y)^T | (I - G Y)^T ] (FP64), and S = F S' F^-1.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "instrument.cuh"

namespace ztoep {
namespace {

__device__ __forceinline__ double2 crecip(double2 z) {
    const double d = z.x * z.x + z.y * z.y;
    return make_double2(z.x / d, -z.y / d);
}

// Y and the elimination array W = [B | C], B = (I + G Y)^T, C = (I - G Y)^T.
__global__ void k_port_setup(const double2 *__restrict__ I, int64_t n, const int *__restrict__ port,
                             const double *__restrict__ len, const double *__restrict__ z0, int p, double2 *Y,
                             double2 *W) {
    const int64_t total = (int64_t)p * p;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / p), k = (int)(idx - (int64_t)a * p);
        const double2 c = I[(int64_t)k * n + port[a]];
        const double sc = 1.0 / (len[a] * len[k]);
        const double2 y = make_double2(c.x * sc, c.y * sc);
        Y[idx] = y;
        const double d = a == k ? 1.0 : 0.0;
        const double2 gy = make_double2(z0[a] * y.x, z0[a] * y.y);  // (G Y)[a][k]
        W[(int64_t)k * 2 * p + a] = make_double2(d + gy.x, gy.y);
        W[(int64_t)k * 2 * p + p + a] = make_double2(d - gy.x, -gy.y);
    }
}

// Step k, one CTA: pivot row = argmax_{i >= k} |W[i][k]| (ties: lowest i),
// swap it into row k, then prow = W[k][:] / W[k][k] and col = W[:][k].  A zero
// or non-finite pivot sets *err.
__global__ void __launch_bounds__(1024) k_gj_pivot(double2 *W, int p, int k, double2 *col, double2 *prow, int *err) {
    __shared__ double s_v[32];
    __shared__ int s_i[32];
    __shared__ int s_piv;
    const int w2 = 2 * p;
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
__global__ void k_gj_elim(double2 *W, int p, int k, const double2 *__restrict__ col, const double2 *__restrict__ prow) {
    const int w2 = 2 * p;
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

// S[a][k] = F_a S'[a][k] / F_k = sqrt(z0_k / z0_a) X[k][a], X = S'^T.
__global__ void k_port_finish(const double2 *__restrict__ W, const double *__restrict__ z0, int p, double2 *S) {
    const int64_t total = (int64_t)p * p;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(idx / p), k = (int)(idx - (int64_t)a * p);
        const double f = sqrt(z0[k] / z0[a]);
        const double2 x = W[(int64_t)k * 2 * p + p + a];
        S[idx] = make_double2(f * x.x, f * x.y);
    }
}

unsigned grid_for_elems(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace
}  // namespace ztoep

using namespace ztoep;

extern "C" ztoep_status_t ztoep_port_matrices(int32_t p, int64_t n, const void *I, const int32_t *ports,
                                              const double *edge_len, const double *z0, void *Y, void *S,
                                              void *stream) {
    if (p < 1 || p > 16384 || n < 1 || !I || !ports || !edge_len || !z0 || !Y || !S || Y == S || Y == I || S == I)
        return ZTOEP_ERR_ARG;
    for (int a = 0; a < p; ++a)
        if (ports[a] < 0 || ports[a] >= n || !(edge_len[a] > 0.0) || !std::isfinite(edge_len[a]) || !(z0[a] > 0.0) ||
            !std::isfinite(z0[a]))
            return ZTOEP_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t wbytes = sizeof(double2) * (size_t)p * 2 * p;
    const size_t small = sizeof(double2) * (size_t)3 * p + sizeof(double) * 2 * p + sizeof(int) * (p + 1);
    unsigned char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, wbytes + small + 64, s) != cudaSuccess) {
        cudaGetLastError();
        return ZTOEP_ERR_NOMEM;
    }
    double2 *W = reinterpret_cast<double2 *>(buf);
    double2 *col = W + (size_t)p * 2 * p;
    double2 *prow = col + p;
    double *dlen = reinterpret_cast<double *>(prow + 2 * p);
    double *dz0 = dlen + p;
    int *dport = reinterpret_cast<int *>(dz0 + p);
    int *derr = dport + p;
    ztoep_status_t st = ZTOEP_OK;
    int herr = 0;
    auto run = [&]() -> ztoep_status_t {
        ZT_CUDA(cudaMemcpyAsync(dlen, edge_len, sizeof(double) * p, cudaMemcpyHostToDevice, s));
        ZT_CUDA(cudaMemcpyAsync(dz0, z0, sizeof(double) * p, cudaMemcpyHostToDevice, s));
        ZT_CUDA(cudaMemcpyAsync(dport, ports, sizeof(int) * p, cudaMemcpyHostToDevice, s));
        ZT_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), s));
        {
            KScope ks(K_MISC, s);
            k_port_setup<<<grid_for_elems((int64_t)p * p), 256, 0, s>>>(static_cast<const double2 *>(I), n, dport,
                                                                        dlen, dz0, p, static_cast<double2 *>(Y), W);
            ZT_CUDA(cudaGetLastError());
        }
        const int pt = std::min(1024, std::max(32, (p + 31) / 32 * 32));
        for (int k = 0; k < p; ++k) {
            KScope ks(K_MISC, s);
            ks.add(2);
            k_gj_pivot<<<1, pt, 0, s>>>(W, p, k, col, prow, derr);
            k_gj_elim<<<grid_for_elems((int64_t)p * 2 * p), 256, 0, s>>>(W, p, k, col, prow);
            ZT_CUDA(cudaGetLastError());
        }
        {
            KScope ks(K_MISC, s);
            k_port_finish<<<grid_for_elems((int64_t)p * p), 256, 0, s>>>(W, dz0, p, static_cast<double2 *>(S));
            ZT_CUDA(cudaGetLastError());
        }
        ZT_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
        return ZTOEP_OK;
    };
    st = run();
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ZTOEP_ERR_CUDA;
    if (st != ZTOEP_OK) return st;
    return herr ? ZTOEP_ERR_NONFINITE : ZTOEP_OK;
}
