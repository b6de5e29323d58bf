// Level-1 solve by the Schur complement (Sec. II-D, Eqs. solveEqSystem1/2):
// with Z = [[A, B^T], [B, C]] and a plan of A alone,
//   A F = B^T          (E right-hand sides: the rows of B)
//   A U = V_T          (the Toeplitz part of each right-hand side)
//   S   = C - B F      (E x E Schur complement)
//   I_E = S^-1 (V_E - B U)
//   I_T = U - F I_E.
// The paper states the outer step for V_E = 0; V_E is kept general here.
// The A-solves are the batched GMRES of ztoep_solve (chunks of up to 256
// RHS, the tensor-core product range); the three contractions over N_T or E
// are an FP64 complex tiled kernel; S is solved by FP64 Gauss-Jordan.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "gj.cuh"
#include "instrument.cuh"

namespace ztoep {
namespace {

// Out(i, j) = D(i, j) - sum_k P(i, k) Q(k, j) for i < ni, j < nj, k < nk, every
// operand addressed by its own (row, column) strides (D may be null: 0).  A
// CTA of 16 x 16 threads forms a 32 x 32 tile, 2 x 2 outputs per thread, with
// K in chunks of 16 staged in shared memory; each operand tile is loaded with
// its unit-stride index fastest.  Sums run over k in a fixed order.
struct Mat {
    const double2 *p;
    int64_t si, sj;
};
__global__ void __launch_bounds__(256) k_zgemm_sub(Mat P, Mat Q, Mat D, double2 *out, int64_t oi, int64_t oj, int ni,
                                                   int nj, int64_t nk) {
    __shared__ double2 sp[32][17], sq[16][33];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    double2 acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[a][c] = make_double2(0.0, 0.0);
    const bool p_ifast = P.si == 1, q_jfast = Q.sj == 1;
    for (int64_t k0 = 0; k0 < nk; k0 += 16) {
        for (int e = threadIdx.x; e < 512; e += 256) {  // P tile: 32 i x 16 k
            const int ii = p_ifast ? (e & 31) : (e >> 4), kk = p_ifast ? (e >> 5) : (e & 15);
            const int i = i0 + ii;
            const int64_t k = k0 + kk;
            sp[ii][kk] = (i < ni && k < nk) ? P.p[i * P.si + k * P.sj] : make_double2(0.0, 0.0);
        }
        for (int e = threadIdx.x; e < 512; e += 256) {  // Q tile: 16 k x 32 j
            const int jj = q_jfast ? (e & 31) : (e >> 4), kk = q_jfast ? (e >> 5) : (e & 15);
            const int j = j0 + jj;
            const int64_t k = k0 + kk;
            sq[kk][jj] = (j < nj && k < nk) ? Q.p[k * Q.si + j * Q.sj] : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const double2 p0 = sp[ty][kk], p1 = sp[ty + 16][kk];
            const double2 q0 = sq[kk][tx], q1 = sq[kk][tx + 16];
            acc[0][0] = cfma(p0, q0, acc[0][0]);
            acc[0][1] = cfma(p0, q1, acc[0][1]);
            acc[1][0] = cfma(p1, q0, acc[1][0]);
            acc[1][1] = cfma(p1, q1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * c;
            if (i < ni && j < nj) {
                const double2 d = D.p ? D.p[i * D.si + j * D.sj] : make_double2(0.0, 0.0);
                out[i * oi + j * oj] = d - acc[a][c];
            }
        }
}

// B with the columns of absent elements zeroed (the masked system's B M).
__global__ void k_mask_cols(const double2 *__restrict__ B, const uint8_t *__restrict__ active, double2 *Bm,
                            int64_t NT, int b, int64_t total) {
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx % NT;
        Bm[idx] = active[t / b] ? B[idx] : make_double2(0.0, 0.0);
    }
}

ztoep_status_t zgemm_sub(Mat P, Mat Q, Mat D, double2 *out, int64_t oi, int64_t oj, int ni, int nj, int64_t nk,
                         cudaStream_t s) {
    KScope ks(K_MISC, s);
    const dim3 grid((nj + 31) / 32, (ni + 31) / 32);
    if (grid.y > 65535) return ZTOEP_ERR_UNSUPPORTED;
    k_zgemm_sub<<<grid, 256, 0, s>>>(P, Q, D, out, oi, oj, ni, nj, nk);
    ZT_CUDA(cudaGetLastError());
    return ZTOEP_OK;
}

}  // namespace
}  // namespace ztoep

using namespace ztoep;

extern "C" ztoep_status_t ztoep_solve_schur(ztoep_plan_t pa, int32_t n_edge, const void *B, const void *C,
                                            const ztoep_solve_opts_t *o, int32_t nrhs, const void *V, void *X,
                                            ztoep_solve_info_t *info, void *stream) {
    if (!pa || !o || n_edge < 1 || n_edge > 16384 || !B || !C || nrhs < 1 || !V || !X || V == X) return ZTOEP_ERR_ARG;
    ztoep_plan_info_t pi{};
    ZT_TRY(ztoep_plan_get_info(pa, &pi));
    if (pi.n_edge != 0) return ZTOEP_ERR_ARG;  // the plan must be of A alone
    const int64_t NT = pi.n, E = n_edge, N = NT + E;
    cudaStream_t s = (cudaStream_t)stream;
    const int wq = (int)E + nrhs;  // [S | R]
    const size_t fbytes = sizeof(double2) * (size_t)E * NT, ubytes = sizeof(double2) * (size_t)nrhs * NT;
    const size_t wbytes = sizeof(double2) * (size_t)E * wq;
    const size_t small = sizeof(double2) * (size_t)(E + wq) + 64;
    const size_t mbytes = pa->masked ? fbytes : 0;  // B M for a masked grid
    unsigned char *buf = nullptr;
    if (cudaMallocAsync((void **)&buf, fbytes + 2 * ubytes + wbytes + small + mbytes, s) != cudaSuccess) {
        cudaGetLastError();
        return ZTOEP_ERR_NOMEM;
    }
    double2 *F = reinterpret_cast<double2 *>(buf);  // rows: A^-1 B[e]^T
    double2 *Vt = F + (size_t)E * NT;               // [nrhs][NT] Toeplitz part of V
    double2 *U = Vt + (size_t)nrhs * NT;            // A^-1 V_T
    double2 *W = U + (size_t)nrhs * NT;             // [E][E + nrhs]
    double2 *col = W + (size_t)E * wq;
    double2 *prow = col + E;
    int *derr = reinterpret_cast<int *>(prow + wq);
    double2 *Bm = pa->masked ? reinterpret_cast<double2 *>(buf + fbytes + 2 * ubytes + wbytes + small) : nullptr;
    const double2 *Bd = static_cast<const double2 *>(B), *Cd = static_cast<const double2 *>(C);
    const double2 *Vd = static_cast<const double2 *>(V);
    double2 *Xd = static_cast<double2 *>(X);
    int herr = 0;
    ztoep_status_t worst = ZTOEP_OK;
    auto run = [&]() -> ztoep_status_t {
        ZT_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), s));
        if (Bm) {  // absent elements: identity rows and columns, so B's columns there are dropped
            KScope ks(K_MISC, s);
            const int64_t total = E * NT;
            k_mask_cols<<<(unsigned)std::min<int64_t>((total + 255) / 256, 8192), 256, 0, s>>>(Bd, pa->active, Bm, NT,
                                                                                               pa->b, total);
            ZT_CUDA(cudaGetLastError());
            Bd = Bm;
        }
        // A F = B^T, in chunks of up to 256 RHS
        std::vector<ztoep_solve_info_t> fi(256);
        for (int64_t e0 = 0; e0 < E; e0 += 256) {
            const int k = (int)std::min<int64_t>(256, E - e0);
            const ztoep_status_t st = ztoep_solve(pa, o, k, Bd + e0 * NT, F + e0 * NT, fi.data(), stream);
            if (st != ZTOEP_OK && st != ZTOEP_ERR_NOCONV && st != ZTOEP_ERR_TIMEOUT) return st;
            if (st != ZTOEP_OK) worst = st;
        }
        // A U = V_T
        ZT_CUDA(cudaMemcpy2DAsync(Vt, sizeof(double2) * NT, Vd, sizeof(double2) * N, sizeof(double2) * NT, nrhs,
                                  cudaMemcpyDeviceToDevice, s));
        {
            const ztoep_status_t st = ztoep_solve(pa, o, nrhs, Vt, U, info, stream);
            if (st != ZTOEP_OK && st != ZTOEP_ERR_NOCONV && st != ZTOEP_ERR_TIMEOUT) return st;
            if (st != ZTOEP_OK) worst = st;
        }
        // S = C - B F  (i = e, j = e', k = t)  -> W[:, 0:E]
        ZT_TRY(zgemm_sub(Mat{Bd, NT, 1}, Mat{F, 1, NT}, Mat{Cd, E, 1}, W, wq, 1, (int)E, (int)E, NT, s));
        // R = V_E - B U  (i = e, j = r, k = t)  -> W[:, E:E+nrhs]
        ZT_TRY(zgemm_sub(Mat{Bd, NT, 1}, Mat{U, 1, NT}, Mat{Vd + NT, 1, N}, W + E, wq, 1, (int)E, nrhs, NT, s));
        ZT_TRY(gj_solve(W, (int)E, wq, col, prow, derr, s));
        // I_T = U - F I_E  (i = r, j = t, k = e): P(r, e) = W[e][E + r], Q(e, t) = F[e][t]
        ZT_TRY(zgemm_sub(Mat{W + E, 1, wq}, Mat{F, NT, 1}, Mat{U, NT, 1}, Xd, N, 1, nrhs, (int)NT, E, s));
        // I_E: X[r][NT + e] = W[e][E + r]  (i = r, j = e, no sum: D only, nk = 0)
        ZT_TRY(zgemm_sub(Mat{W, 0, 0}, Mat{W, 0, 0}, Mat{W + E, 1, wq}, Xd + NT, N, 1, nrhs, (int)E, 0, s));
        ZT_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
        return ZTOEP_OK;
    };
    const ztoep_status_t st = run();
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return ZTOEP_ERR_CUDA;
    if (st != ZTOEP_OK) return st;
    if (herr) return ZTOEP_ERR_NONFINITE;
    return worst;
}
