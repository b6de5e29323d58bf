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
#include "gj.cuh"
#include "instrument.cuh"

namespace ztoep {
namespace {

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
        ZT_TRY(gj_solve(W, p, 2 * p, col, prow, derr, s));
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
