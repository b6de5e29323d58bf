// Far field of the element currents (Sec. III, Eqs. farfieldBasis and
// tensorProd) on the array-factor grid of the plan's embedding.
//
// For the element component the parts are the active elements p = (m, n) at
// offsets d_p = (m a, n a, 0), and the contraction over parts and basis
// functions is
//   F[r][f][t] = -j k eta sum_i Fh[f][t][i] sum_{m,n} e^{j k r^_f . d_p} I[r][(n nx + m) b + i].
// On the directions with k a u = 2 pi kx / lx and k a v = 2 pi ky / ly
// (f = ky lx + kx) the inner sum over the parts is the 2-D DFT the product's
// forward passes compute, at the mirrored frequency (the phase has the
// opposite sign): sum_{m,n} e^{+2 pi i (kx m / lx + ky n / ly)} I = X^[-f].  So
// the far field is the plan's FP64 forward spectrum followed by one b-term
// dot product per (frequency, polarisation, RHS).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "instrument.cuh"

namespace ztoep {
namespace {

// One warp per (f, t, r): out[r][f][t] = c sum_i Fh[f][t][i] Xh[-f][r][i].
__global__ void __launch_bounds__(256) k_far_contract(const double2 *__restrict__ Xh, const double2 *__restrict__ Fh,
                                                      double2 *__restrict__ out, int lx, int ly, int b, int nrhs,
                                                      int npol, double2 c) {
    const int64_t F = (int64_t)lx * ly;
    const int64_t total = F * npol * nrhs;
    const int lane = threadIdx.x & 31;
    for (int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wid < total;
         wid += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int r = (int)(wid % nrhs);
        const int64_t ft = wid / nrhs;
        const int t = (int)(ft % npol);
        const int64_t f = ft / npol;
        const int kx = (int)(f % lx), ky = (int)(f / lx);
        const int64_t fl = (int64_t)((ly - ky) % ly) * lx + (lx - kx) % lx;
        const double2 *fh = Fh + (f * npol + t) * b;
        const double2 *xh = Xh + (fl * nrhs + r) * b;
        double2 acc = make_double2(0.0, 0.0);
        for (int i = lane; i < b; i += 32) acc = cfma(fh[i], xh[i], acc);
        for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        }
        if (lane == 0) out[((int64_t)r * F + f) * npol + t] = cmul(c, acc);
    }
}

}  // namespace
}  // namespace ztoep

using namespace ztoep;

extern "C" ztoep_status_t ztoep_far_field_grid(ztoep_plan_t p, int32_t nrhs, const void *I, int32_t npol,
                                               const void *Fh, double k, double eta, void *F, void *stream) {
    if (!p || !I || !Fh || !F || nrhs < 1 || npol < 1 || npol > 16 || F == I || !std::isfinite(k) ||
        !std::isfinite(eta))
        return ZTOEP_ERR_ARG;
    std::lock_guard<std::mutex> lk(p->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t xbytes = sizeof(double2) * (size_t)p->F * nrhs * p->b;
    double2 *Xh = nullptr;
    if (cudaMallocAsync((void **)&Xh, xbytes, s) != cudaSuccess) {
        cudaGetLastError();
        return ZTOEP_ERR_NOMEM;
    }
    ztoep_status_t st = run_forward_spectrum<double>(p, nrhs, static_cast<const double2 *>(I), Xh, s);
    if (st == ZTOEP_OK) {
        KScope ks(K_MISC, s);
        const int64_t warps = (int64_t)p->F * npol * nrhs;
        const unsigned grid = (unsigned)std::min<int64_t>((warps + 7) / 8, 8LL * p->nsm * 8);
        k_far_contract<<<grid, 256, 0, s>>>(Xh, static_cast<const double2 *>(Fh), static_cast<double2 *>(F), p->lx,
                                            p->ly, p->b, nrhs, npol, make_double2(0.0, -k * eta));
        if (cudaGetLastError() != cudaSuccess) st = ZTOEP_ERR_CUDA;
    }
    cudaFreeAsync(Xh, s);
    return st;
}
