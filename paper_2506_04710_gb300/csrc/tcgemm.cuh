// Batched complex GEMM on tcgen05 tensor cores (3xTF32, FP32 accumulate):
//   C_p[m][q] = sum_k A_p[m][k] X_p[q][k]
// A: complex row-major (k contiguous), lda; X: complex [q][k], ldx.
// C element (q, m) of problem p and K split s lives at
//   C + p * strideC + s * strideCk + q * ldc_q + m * ldc_m.
#pragma once

#include "common.cuh"

namespace ztoep {

struct CgemmArgs {
    const float2 *A;
    int64_t lda, strideA;
    const float2 *X;
    int64_t ldx, strideX;
    float2 *C;
    int64_t ldc_q, ldc_m, strideC, strideCk;
    int M, K, N;     // complex sizes; N <= 256
    int kchunk;      // complex k per CTA (0 = all of K); partial sums per split
    int np, tmem_cols, nraw;  // set by the launcher
    int *err;        // device error word (bounded waits)
};

size_t cgemm_smem_bytes(int np);
bool cgemm_fits(int n);  // a GEMM with n right-hand sides fits in shared memory
ztoep_status_t launch_cgemm_tc(CgemmArgs g, int nprob, cudaStream_t s);
// Warp-specialised persistent variant (TMA operand loads, double-buffered
// accumulators); UNSUPPORTED when the operands do not suit TMA.
ztoep_status_t launch_cgemm_tc2(const CgemmArgs &g, int nprob, int nsm, cudaStream_t s);
// The pipelined kernel when it applies, else the lock-step one.
inline ztoep_status_t launch_cgemm(const CgemmArgs &g, int nprob, int nsm, cudaStream_t s) {
    const ztoep_status_t st = launch_cgemm_tc2(g, nprob, nsm, s);
    return st == ZTOEP_ERR_UNSUPPORTED ? launch_cgemm_tc(g, nprob, s) : st;
}

// Number of K splits the launcher uses for a given K and chunk.
inline int cgemm_splits(int K, int kchunk) {
    const int kc = (kchunk + 15) / 16 * 16;
    return (K + kc - 1) / kc;
}

}  // namespace ztoep
