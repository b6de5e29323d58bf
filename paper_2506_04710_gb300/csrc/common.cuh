// Internal definitions shared by the ztoep CUDA translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <mutex>

#include "ztoep.h"

namespace ztoep {

// ---------------------------------------------------------------- complex
template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };
template <typename R> using cplx_t = typename Cplx<R>::T;

__host__ __device__ __forceinline__ float2 mkc(float r, float i) { return make_float2(r, i); }
__host__ __device__ __forceinline__ double2 mkc(double r, double i) { return make_double2(r, i); }

template <typename C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }

__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// a * b
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
// acc + a * b
__host__ __device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}
__host__ __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
    return acc;
}
// acc + conj(a) * b
__host__ __device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 acc) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
    return acc;
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
// |a|^2 as one explicit fused multiply-add, so that the compiler cannot
// contract it (or a sum it is added to) differently where it is inlined: the
// same value in every kernel.
__host__ __device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }

// a / b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962).
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    if (fabs(b.x) >= fabs(b.y)) {
        double r = b.y / b.x, d = b.x + b.y * r;
        return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    double r = b.x / b.y, d = b.x * r + b.y;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

template <typename Dst, typename Src> __host__ __device__ __forceinline__ Dst ccast(Src s) {
    Dst d; d.x = s.x; d.y = s.y; return d;
}

// ---------------------------------------------------------------- FFT plan
// Radix decomposition of one transform length (radices 2, 3, 4, 5).
struct Fft1D {
    int L;
    int nst;
    int rad[12];
    // per stage: the sub-transform length Ns entering it and M = 65536 / Ns + 1,
    // so that j / Ns == (j * M) >> 16 for every j < 256 (j < L / radix here)
    int ns[12], mag[12];
};

// Radix sequence for length L: order 0 takes radix 4 first (then 2, 3, 5),
// order 1 the reverse sequence.
Fft1D make_fft1d(int L, int order = 0);
int smooth_size_at_least(int n);
bool is_smooth(int n);

// ---------------------------------------------------------------- plan
// Launch and layout choices of a plan; -1 / 0 = the built-in heuristic.  Set
// when the plan is built (by the autotuner or from its cache) and fixed for the
// plan's life, so every solve on it sums in the same order whatever its RHS
// count.  The FFT-pass knobs apply to FP32 products; their values do not
// change the arithmetic of a line's transform.
struct TuneParams {
    int rad_order[2] = {0, 0};  // radix order of the x and y transforms (plan and products)
    int lib[2] = {-1, -1};      // log2 channels per CTA of the FP32 x / y passes
    int thr[2] = {0, 0};        // threads per CTA of the FP32 x / y passes (shared-memory kernel)
    int fk[2] = {0, 0};         // FP32 x / y pass kernel: 0 register where the length allows, 1 shared memory, 2 register
    int bp_split = 0;           // threads per dot product in the SIMT block product
    int bp_per_sm = 0;          // block-product CTAs per SM
    int tc_kchunk = 0;          // K per CTA of the tensor-core B x_T product
};

struct MatvecWs {  // per-precision matvec workspace, sized for `cap` RHS
    int cap = 0;
    void *xin = nullptr;    // [cap][N] input copy in this precision (public matvec / solver)
    void *yout = nullptr;   // [cap][N] output in this precision
    void *X1 = nullptr;     // [cap][ny][lx][b] after the x pass (also reused by the inverse y pass)
    void *Xh = nullptr;     // [F][cap][b] spectrum (block product runs in place)
    void *ET = nullptr;     // [nsplit][cap][NT] B^T x_E partial sums
    void *Ep = nullptr;     // B x_T partial sums: k_edge3 [cap][E][ntile], else [ntile or K split][cap][E]
    void *Yh = nullptr;     // [F][cap][b] out-of-place block-product output (tensor path, side plans)
    void *Ps = nullptr;     // [blocks][4k][cap][Lmax] partials of B x_T along each side, frequency domain
    void *Us = nullptr;     // [cap][4k][Lmax] DFTs of the side slices of x_E
    size_t bytes = 0;
};

struct SolveWs {  // Krylov workspace, sized for `cap` RHS and restart `m`
    int cap = 0, m = 0;
    double2 *Vb = nullptr;     // [(m+1)][cap][N] unnormalised Krylov basis
    double2 *w = nullptr;      // [cap][N] FP64 product output
    double2 *xin64 = nullptr;  // [cap][N] FP64 product input (next basis vector)
    double2 *vbuf = nullptr;   // [cap][N] right-hand sides (graph-owned copy)
    double2 *xbuf = nullptr;   // [cap][N] iterate (graph-owned copy)
    double2 *rbuf = nullptr;   // [cap][N] FP64 true residual of the current sweep
    double2 *dbuf = nullptr;   // [cap][N] correction accumulated over the sweep's restarts
    double2 *H = nullptr;      // [cap][m+1][m] Hessenberg (rotated to R)
    double2 *cs = nullptr;     // [cap][m]
    double2 *sn = nullptr;     // [cap][m]
    double2 *g = nullptr;      // [cap][m+1]
    double2 *h1 = nullptr;     // [cap][m+1]
    double2 *h2 = nullptr;     // [cap][m+1]
    double2 *part = nullptr;   // [cap][rows][m+2] chunk partial sums and inner nodes of the reduction tree
    double *nrm = nullptr;     // [cap][8] scalars, then [cap][m+1] basis norms
    int *st = nullptr;         // [cap][8] per-RHS state
    unsigned *cnt = nullptr;   // [cap][cstride] last-arriver tickets of the cross-CTA sums
    void *ctl = nullptr;       // device solve control block
    int cstride = 0;           // reduction tickets per RHS
    int *hst = nullptr;        // host pinned mirror of st (+ control words)
    double *hnrm = nullptr;    // host pinned mirror of nrm
    size_t bytes = 0;
};

// One instantiated solve graph (per precision, RHS count and restart length).
struct SolveGraph {
    int prec = -1, nrhs = 0, m = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t k_fixed = 0, k_sweep = 0, k_restart = 0, k_iter = 0, k_first_product = 0, k_reorth = 0;  // kernels per part
};

struct PlanImpl;

}  // namespace ztoep

struct ztoep_plan_s {
    int nx = 0, ny = 0, b = 0, E = 0, lx = 0, ly = 0, F = 0;
    int64_t NT = 0, N = 0;
    int npairs = 0;
    int device = 0;
    int nsm = 0;
    int l2_bytes = 0;  // device L2 capacity (cache-hint choices)
    bool masked = false;
    ztoep::Fft1D fx{}, fy{};
    ztoep::TuneParams tune;
    int2 *pairs = nullptr;          // [npairs] (f, -f); f == -f for self-paired frequencies
    int *rep = nullptr;             // [F] pair index of f if f is the stored one, else -1-pair
    double2 *That64 = nullptr;      // [npairs][b][b]
    float2 *That32 = nullptr;
    double2 *B64 = nullptr;         // [E][NT], absent elements' columns zero
    float2 *B32 = nullptr;          // [E][ldb32] = [B | C | 0] (FP32 edge kernel reads one row for y_E)
    double2 *C64 = nullptr;         // [E][E]
    float2 *C32 = nullptr;
    float2 *That32full = nullptr;   // [F][b][b] every frequency, for the tensor-core product
    float2 *B32T = nullptr;         // [NT][E] transposed B, for the tensor-core B^T x_E
    int side_k = 0;                 // > 0: perimeter side-Toeplitz B, k edge unknowns per cell side
    double2 *G64 = nullptr;         // [4k][F][b] 2-D spectra of the side generators (replace B)
    float2 *G32 = nullptr;
    size_t tc_bytes = 0;
    uint8_t *active = nullptr;      // [ny*nx] device copy, nullptr if all active
    double2 *twx64 = nullptr, *twy64 = nullptr;  // exp(-2 pi i t / L)
    float2 *twx32 = nullptr, *twy32 = nullptr;
    int *err = nullptr;             // device error word (bounded waits)
    size_t resident = 0;
    ztoep::MatvecWs ws32, ws64;
    ztoep::SolveWs sws;
    ztoep::SolveGraph graphs[4];    // small cache of instantiated solve graphs
    int graph_next = 0;
    cudaStream_t side = nullptr;    // edge-coupling branch of the matvec
    cudaStream_t aux = nullptr;     // solve graph branch beside the product (Givens rotations of the last column)
    cudaStream_t cap = nullptr;     // stream used to capture solve graphs
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_et = nullptr;    // edge branch: B^T x_E complete (the rest of the branch may still run)
    std::mutex mu;
};

namespace ztoep {

#define ZT_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return ZTOEP_ERR_CUDA;      \
    } while (0)

#define ZT_TRY(call)                                       \
    do {                                                   \
        ztoep_status_t s_ = (call);                        \
        if (s_ != ZTOEP_OK) return s_;                     \
    } while (0)

ztoep_status_t dalloc(void **p, size_t bytes, size_t *acc);
// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
inline bool bytes_overlap(const void *a, size_t na, const void *b, size_t nb) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}
// Build a plan with the given launch/layout choices (ztoep_plan uses the defaults).
ztoep_status_t plan_create(const ztoep_desc_t *d, const void *T, const void *B, const void *C, cudaStream_t s,
                           const TuneParams &tp, ztoep_plan_t *out);
void free_solve_graphs(ztoep_plan_t p);  // cached graphs bake in workspace pointers

// Matvec in one precision on plan-internal buffers: y = Z' x, x/y [nrhs][N].
template <typename R>
ztoep_status_t run_matvec(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *y,
                          cudaStream_t s);
template <typename R> ztoep_status_t ensure_ws(ztoep_plan_t p, int nrhs);
// Tensor-core operands (full FP32 spectrum, transposed B) for FP32 products
// with at least kTcMinRhs right-hand sides.
constexpr int kTcMinRhs = 16;
constexpr int kTcMaxRhs = 256;
ztoep_status_t ensure_tensor_data(ztoep_plan_t p, int nrhs, cudaStream_t s);
// Perimeter side-Toeplitz edge coupling (sides.cu): plan-time generator
// spectra from B; per product: DFTs of the side slices of x_E (sides_uhat),
// after the block product one pass over the spectra that adds the B^T x_E
// terms to Y^ and leaves the partials of B x_T (sides_fused), and y_E from
// those partials and C (sides_finish).  sides_partials: partial-sum elements
// per RHS.
ztoep_status_t sides_build(ztoep_plan_t p, const double2 *B, cudaStream_t s, size_t *acc);
template <typename R>
ztoep_status_t sides_uhat(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, MatvecWs &w, cudaStream_t s);
template <typename R>
ztoep_status_t sides_fused(ztoep_plan_t p, int nrhs, const cplx_t<R> *Xh, cplx_t<R> *Yh, MatvecWs &w,
                           cudaStream_t s);
template <typename R>
ztoep_status_t sides_finish(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *y, MatvecWs &w,
                            cudaStream_t s);
int64_t sides_partials(ztoep_plan_t p);
template <typename R> MatvecWs &ws_of(ztoep_plan_t p);
template <typename R>
ztoep_status_t run_forward_spectrum(ztoep_plan_t p, int nrhs, const cplx_t<R> *x, cplx_t<R> *Xh,
                                    cudaStream_t s);

// Elementwise helpers (kernels in matvec.cu).
ztoep_status_t launch_c128_to_c64(const double2 *src, float2 *dst, int64_t n, cudaStream_t s);
ztoep_status_t launch_c64_to_c128(const float2 *src, double2 *dst, int64_t n, cudaStream_t s);

}  // namespace ztoep
