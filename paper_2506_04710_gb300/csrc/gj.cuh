// FP64 complex Gauss-Jordan elimination with partial pivoting on the device
// (used by the port matrices and the Schur-complement solve).
#pragma once
#include "common.cuh"

namespace ztoep {

// Solves M X = R in place on the p x w row-major array W = [M | R]
// (w >= p): after the p steps the left block is the identity and the right
// block holds X.  col [p] and prow [w] are scratch; *err is set (bit 0) on a
// zero or non-finite pivot.  Two launches per column on stream s.
ztoep_status_t gj_solve(double2 *W, int p, int w, double2 *col, double2 *prow, int *err, cudaStream_t s);

}  // namespace ztoep
