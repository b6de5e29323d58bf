/*
 * ztoep -- solver for the two-level block-Toeplitz method-of-moments systems
 * of finite antenna arrays with electrically connected elements (array
 * decomposition into nine components; Akerstedt, Hultin & Jonsson).
 *
 * The system is Z I = V (Sec. II, Eq. MoMMatrixEq) with
 *
 *     Z = [[A, B^T],
 *          [B, C  ]]                                  (Sec. II-C, Eq. matrixForm)
 *
 * A couples the element (component 5) parts and is two-level block Toeplitz
 * (Eq. submatrixAA): its b x b block for element pair ((m,n),(m',n')) is the
 * generating block T[m-m', n-n'], so it is stored as its (2Nx-1)(2Ny-1)
 * generating blocks.  B couples the E non-Toeplitz edge/margin unknowns to
 * the element unknowns and C couples them among themselves (Sec. II-C, the
 * B and C blocks); both are taken dense here.  Z is symmetric (Sec. II-A), so
 * T[-p,-q] = T[p,q]^T must hold for the input blocks.
 *
 * The product with A is done by embedding the generating blocks in a
 * block circulant of size Lx x Ly >= (2Nx-1) x (2Ny-1), a 2-D FFT over the
 * element indices (m, n), a b x b block product per frequency, an inverse
 * FFT and a crop (the FFT acceleration of Toeplitz products cited in Sec. I);
 * the edge unknowns are coupled in by a separate product with B, B^T and C.
 * Solves are batched restarted GMRES (Sec. II-D names GMRES for the
 * second Toeplitz level) inside an FP64 iterative-refinement loop.
 *
 * Conventions for every entry point:
 *  - Unknown order: Toeplitz unknown (m, n, i), element column m < Nx, row
 *    n < Ny, local basis i < b, has index (n*Nx + m)*b + i (components
 *    indexed bottom-left first, x fastest, Sec. II-C); the E edge unknowns
 *    follow at N_T .. N_T+E-1, N_T = Nx*Ny*b, N = N_T + E.
 *  - Complex numbers are interleaved (re, im) IEEE doubles (complex128)
 *    unless stated otherwise.  Vectors are stored one RHS after the other:
 *    X[r*N + k].
 *  - Device pointers are caller-owned CUDA global memory on the current
 *    device; all work is ordered on the caller's stream (a cudaStream_t
 *    passed as void*, NULL = legacy default stream).  A plan is used by one
 *    stream at a time.
 *  - Errors are returned as status codes; nothing is thrown across the ABI.
 *    ZTOEP_ERR_CUDA means a CUDA call failed (the CUDA error is not
 *    cleared); ZTOEP_ERR_TIMEOUT means a bounded device-side wait gave up.
 */
#ifndef ZTOEP_H
#define ZTOEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ZTOEP_API __attribute__((visibility("default")))
#else
#define ZTOEP_API
#endif

typedef struct ztoep_plan_s *ztoep_plan_t;

typedef enum {
    ZTOEP_OK = 0,
    ZTOEP_ERR_ARG = 1,          /* invalid argument or descriptor */
    ZTOEP_ERR_NOMEM = 2,        /* device allocation failed or footprint cap exceeded */
    ZTOEP_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    ZTOEP_ERR_NOCONV = 4,       /* iteration limit reached before the tolerance */
    ZTOEP_ERR_TIMEOUT = 5,      /* a bounded device-side wait or the solve timeout expired */
    ZTOEP_ERR_UNSUPPORTED = 6,  /* valid request outside what this build implements */
    ZTOEP_ERR_NONFINITE = 7     /* NaN/Inf in a right-hand side or residual */
} ztoep_status_t;

typedef enum {
    ZTOEP_FP64 = 0,  /* every step in complex FP64 */
    ZTOEP_MIXED = 1  /* FFTs and block/edge products in complex FP32 (inner
                        solves), FP64 residuals, Arnoldi, Givens and updates */
} ztoep_precision_t;

/* Array descriptor.  nx, ny >= 1, b >= 1 (b <= 128), n_edge >= 0.
 * active: HOST pointer to ny*nx bytes (row n, column m at [n*nx + m]),
 *   nonzero = element present; NULL = all present.  An absent element's
 *   unknowns get identity rows and columns, Z' = M Z M + (I - M), so with a
 *   zero right-hand side there the solution there is exactly zero.
 * lx, ly: circulant embedding sizes; 0 = choose automatically (the smallest
 *   size >= 2n-1 whose prime factors are 2, 3 and 5).  Explicit sizes must be
 *   >= 2n-1, <= 256 and have only those prime factors.
 * edge_per_cell: 0 = B is a general dense matrix.  k >= 1 declares the
 *   perimeter layout: n_edge = 2k(nx + ny) edge unknowns, k per cell side,
 *   ordered counter-clockwise from the corner (0, 0) (bottom side left to
 *   right, right side upwards, top side right to left, left side downwards),
 *   so that each side's block of B is one-level block Toeplitz along its side
 *   (the side blocks of Sec. II-C, Eqs. submatrixB12/B34): the entry of edge
 *   unknown (cell c, sub-position s) and element (m, n) depends on c - m (top
 *   and bottom) or c - n (left and right).  The plan then keeps the 2-D spectra
 *   of the 4k side generators instead of B and applies B and B^T in the
 *   frequency domain of the FFT product.  The structure is verified on B at
 *   plan time (relative 1e-11 of max |B|, columns of absent elements
 *   excepted); a B that does not have it is rejected with ARG. */
typedef struct {
    int32_t nx, ny, b, n_edge;
    const uint8_t *active;
    int32_t lx, ly;
    int32_t edge_per_cell;
} ztoep_desc_t;

typedef struct {
    double tol;          /* stop when ||v - Z x||_2 <= tol ||v||_2 for every RHS (true FP64 residual) */
    int32_t restart;     /* GMRES restart length m, 1..128 */
    int32_t max_iter;    /* cap on inner iterations per RHS, summed over cycles */
    int32_t max_outer;   /* cap on refinement sweeps (true-residual evaluations) */
    int32_t prec;        /* ztoep_precision_t */
    double inner_tol;    /* MIXED: relative reduction asked of each inner solve */
    int64_t timeout_ns;  /* wall-clock limit for the whole solve, 0 = none */
    int32_t flags;       /* ZTOEP_FLAG_* bits */
} ztoep_solve_opts_t;

/* Ignore X on entry and start from x = 0 (saves the first FP64 product). */
#define ZTOEP_FLAG_ZERO_GUESS 1
/* Drive the refinement and GMRES loops from the host, one kernel launch at a
 * time, instead of one CUDA graph with conditional nodes (same kernels and
 * results; slower; for profilers that cannot look inside such graphs). */
#define ZTOEP_FLAG_HOST_LOOP 2

typedef struct {
    int32_t outer;        /* true-residual evaluations (refinement sweeps) */
    int32_t inner_iters;  /* Krylov iterations (matrix products) used */
    int32_t status;       /* ztoep_status_t for this RHS */
    int32_t second_passes;  /* Arnoldi steps that took a second Gram-Schmidt pass */
    double rel_residual;  /* final ||v - Z x|| / ||v|| in FP64 */
} ztoep_solve_info_t;

typedef struct {
    int32_t nx, ny, b, n_edge, lx, ly;
    int64_t n_toep, n;          /* N_T and N */
    int64_t n_pairs;            /* stored frequency blocks (f and -f share one, T^(-f) = T^(f)^T) */
    size_t resident_bytes;      /* device bytes held by the plan */
    size_t dense_bytes;         /* bytes the dense complex128 Z would need, N^2 * 16 */
} ztoep_plan_info_t;

/* Defaults: tol 1e-8, restart 30, max_iter 4000, max_outer 100, MIXED,
 * inner_tol 1e-5, no timeout, no flags. */
ZTOEP_API ztoep_status_t ztoep_default_opts(ztoep_solve_opts_t *opts);

/* Build a plan: embed the generating blocks in the Lx x Ly block circulant,
 * FFT them over (m, n) in FP64 (Eq. submatrixAA structure), keep the
 * transformed blocks of one frequency of each pair {f, -f} resident in FP64
 * and FP32, and keep B (absent elements' columns zeroed; or, with
 * desc->edge_per_cell, the spectra of its side generators) and C in FP64 and
 * FP32.
 *   T: device complex128 [2ny-1][2nx-1][b][b]; T[q+ny-1][p+nx-1] is the
 *      block of offset (p, q) = (m-m', n-n').
 *   B: device complex128 [n_edge][N_T] (NULL iff n_edge == 0).
 *   C: device complex128 [n_edge][n_edge] (NULL iff n_edge == 0).
 * The inputs are read on `stream` and may be freed once the stream has
 * passed this call.  *out owns its device memory until ztoep_plan_destroy.
 * Errors: ARG (bad descriptor/pointers), NOMEM, CUDA. */
ZTOEP_API ztoep_status_t ztoep_plan(const ztoep_desc_t *desc, const void *T, const void *B, const void *C,
                          void *stream, ztoep_plan_t *out);

/* Y = Z' X for nrhs right-hand sides (Z' with absent elements masked): the
 * left-hand side of Z I = V (Sec. II, Eq. MoMMatrixEq) with Z in the block
 * form of Sec. II-C, Eq. matrixForm, and its element block A applied through
 * the two-level block-Toeplitz structure of Eq. submatrixAA (circulant
 * embedding, 2-D FFT over the element indices, per-frequency b x b block
 * product, inverse FFT, crop; the FFT acceleration of Sec. I), B, B^T and C
 * applied directly.
 *   X, Y: device complex128 [nrhs][N]; the two byte ranges must not overlap.
 *   prec: ZTOEP_FP64 computes in FP64; ZTOEP_MIXED rounds X to FP32 and
 *   computes the FFTs and products in FP32 (result widened to FP64).
 * Errors: ARG (also for overlapping X and Y), NOMEM (workspace), CUDA. */
ZTOEP_API ztoep_status_t ztoep_matvec(ztoep_plan_t plan, int32_t prec, int32_t nrhs, const void *X, void *Y,
                            void *stream);

/* Edge-coupling part of the FP64 product, allocating nothing.  The paper has
 * no counterpart: this is a service for callers that cannot allocate device
 * memory at call time, such as real-time or embedded hosts that forbid
 * allocation after start-up (an allocation may wait for the whole device or
 * fail under fragmentation at an unpredictable moment) and frameworks whose
 * memory pool has already reserved all device memory.
 *   Y[r][t]       = sum_e B[e][t] x_E[r][e]                 (t < N_T; 0 on absent elements)
 *   Y[r][N_T + e] = sum_t B[e][t] x_T[r][t] + sum_e' C[e][e'] x_E[r][e']
 *   X, Y: device complex128 [nrhs][N]; the two byte ranges must not overlap
 *   (ARG otherwise).  The plan's device must be
 *   current.  The partial sums live in a fixed 16 MiB device array that every
 *   device holding this library keeps until the process exits; nrhs is
 *   limited by it (about 4 for a 32x32 array with b = 64 and 512 edge
 *   unknowns) and a call that would need more returns ZTOEP_ERR_NOMEM without
 *   doing anything.  The first call on a device looks up the array's device
 *   address (cudaGetSymbolAddress); make that first call before any stream
 *   capture.  All calls share the array: calls whose work overlaps on the GPU
 *   (other streams, other threads) race and must be serialised by the caller.
 *   No cudaMalloc, cudaFree or allocating library routine is called.
 * Errors: ARG, NOMEM (scratch cap), CUDA, UNSUPPORTED (device index >= 64,
 * or a plan built with desc->edge_per_cell > 0, which keeps no dense B). */
ZTOEP_API ztoep_status_t ztoep_edge_product_noalloc(ztoep_plan_t plan, int32_t nrhs, const void *X, void *Y,
                                                    void *stream);

/* Solve Z' X = V (Sec. II, Eq. MoMMatrixEq; Z' as for ztoep_matvec) for nrhs
 * right-hand sides by batched restarted GMRES, the iterative solver the paper
 * names for the second Toeplitz level (Sec. II-D), with the FFT products of
 * Sec. I inside an FP64 iterative-refinement loop.
 *   V: device complex128 [nrhs][N].
 *   X: device complex128 [nrhs][N]; initial guess on entry, solution on
 *      exit (on NOCONV/TIMEOUT the best iterate).
 *   info: HOST array of nrhs entries, may be NULL.
 * FP64: restarted GMRES(m) entirely in FP64, restarted on the true residual.
 * MIXED: FP64 refinement x <- x + d, d from a GMRES(m) cycle on Z d = r
 *   with FP32 products and FP64 Arnoldi/Givens/least squares, r = v - Z x in
 *   FP64 between cycles.
 * The whole refinement/GMRES loop runs on the device as one CUDA graph
 * (loops as conditional graph nodes, instantiated once per precision, RHS
 * count and restart length and cached in the plan); V is copied into the
 * plan's buffers first and the solution copied back to X at the end.
 * timeout_ns is enforced on the device (%globaltimer) between iterations.
 * Returns the worst per-RHS status after synchronising `stream` once. */
ZTOEP_API ztoep_status_t ztoep_solve(ztoep_plan_t plan, const ztoep_solve_opts_t *opts, int32_t nrhs,
                           const void *V, void *X, ztoep_solve_info_t *info, void *stream);

/* One solve of `count` independent systems (1..8 plans of any sizes: nx,
 * ny, b, n_edge may all differ), each member exactly as ztoep_solve would
 * solve it alone (the same arithmetic, hence bitwise the same result and
 * info), but as one CUDA graph in which every Arnoldi, residual and update
 * step is a single launch over all members' RHS and the members' products
 * run concurrently (a member with no RHS left in a cycle skips its product).
 * This serves many small or uneven systems (serving, parameter sweeps) whose
 * separate solves would each be bound by launch latency.
 *   plans: host array [count] of distinct plans on the current device.
 *   opts: one set of options for all members (one control loop).
 *   nrhs: host int32 [count]; V, X: host arrays [count] of device pointers,
 *   V[i], X[i] complex128 [nrhs[i]][N_i] (X[i]: initial guess in, solution out).
 *   info: host array [count] of host arrays [nrhs[i]] (entries may be NULL),
 *   or NULL.
 * The graph is built for the call and released after it (a few ms of host
 * time).  Returns the worst per-RHS status after synchronising `stream`.
 * Errors: ARG (bad counts or pointers, a plan given twice, plans on different
 * devices), UNSUPPORTED (members whose sizes need different chunk shapes:
 * systems above 8 x (SM count) x 256 unknowns cannot be grouped with smaller
 * ones), NOMEM, CUDA; per-RHS NOCONV/TIMEOUT/NONFINITE as ztoep_solve. */
ZTOEP_API ztoep_status_t ztoep_solve_group(int32_t count, const ztoep_plan_t *plans, const ztoep_solve_opts_t *opts,
                                           const int32_t *nrhs, const void *const *V, void *const *X,
                                           ztoep_solve_info_t *const *info, void *stream);

/* ztoep_solve with V and X in HOST memory (pinned or pageable): copies V
 * and the initial guess to the device, solves, copies X back.  The device
 * buffers are the plan's own. */
ZTOEP_API ztoep_status_t ztoep_solve_host(ztoep_plan_t plan, const ztoep_solve_opts_t *opts, int32_t nrhs,
                                const void *V_host, void *X_host, ztoep_solve_info_t *info,
                                void *stream);

/* Forward spectrum of the Toeplitz part of X (inspection of the embedding
 * and FFT stage): Xhat[f][r][i] = sum_{m,n} x[r][(n*nx+m)*b+i] w_Lx^(-kx m)
 * w_Ly^(-ky n), f = ky*lx + kx, absent elements taken as zero.
 *   X: device complex128 [nrhs][N]; Xhat: device complex128 [lx*ly][nrhs][b].
 *   prec as in ztoep_matvec (MIXED computes in FP32, widened on output). */
ZTOEP_API ztoep_status_t ztoep_forward_spectrum(ztoep_plan_t plan, int32_t prec, int32_t nrhs,
                                      const void *X, void *Xhat, void *stream);

/* Copy the plan's FP64 transformed blocks of every frequency into
 * That: device complex128 [ly*lx][b][b] (frequency f = ky*lx + kx), rebuilding
 * the blocks of -f as transposes of the stored ones. */
ZTOEP_API ztoep_status_t ztoep_plan_spectrum(ztoep_plan_t plan, void *That, void *stream);

ZTOEP_API ztoep_status_t ztoep_plan_get_info(ztoep_plan_t plan, ztoep_plan_info_t *info);

/* ---- Port matrices (Sec. IV-B) ----
 * After a solve with the delta excitations V = [e_{i_1}, ..., e_{i_p}]:
 *   I      device complex128 [p][n]: row k is the solution for the excitation
 *          at port k (the layout ztoep_solve writes for p RHS);
 *   ports  host int32 [p]: the unknown indices i_k (0 <= i_k < n);
 *   edge_len host double [p]: the ports' edge lengths l_{i_k} (> 0);
 *   z0     host double [p]: real reference impedances (> 0).
 * Writes (device complex128 [p][p], row-major):
 *   Y = L I^ L, I^[a][k] = I[k][i_a] (port currents), L = diag(1 / l_{i_k});
 *   S = F (Z_port - G)(Z_port + G)^-1 F^-1 with Z_port = Y^-1, G = diag(z0),
 *       F = diag(1 / (2 sqrt(z0))): the power-wave scattering matrix, formed as
 *       F (I - G Y)(I + G Y)^-1 F^-1 by FP64 Gauss-Jordan elimination with
 *       partial pivoting (no inverse of Y).
 * Stream-ordered; returns after the work completes (it reads back a status
 * word).  Allocates 2 p^2 complex128 of stream-ordered workspace.  Errors:
 * ARG (bad sizes or values, Y/S aliasing I or each other), NOMEM,
 * NONFINITE (a zero or non-finite pivot: I + G Y singular), CUDA. */
ZTOEP_API ztoep_status_t ztoep_port_matrices(int32_t p, int64_t n, const void *I, const int32_t *ports,
                                             const double *edge_len, const double *z0, void *Y, void *S,
                                             void *stream);

/* ---- Level-1 solve by the Schur complement (Sec. II-D, Eqs. solveEqSystem1/2) ----
 * Z = [[A, B^T], [B, C]] solved through solves with A alone:
 *   A F = B^T, A U = V_T, S = C - B F, I_E = S^-1 (V_E - B U), I_T = U - F I_E.
 *   plan_A: a plan of the same Toeplitz blocks with n_edge = 0 (ARG otherwise);
 *   B: device complex128 [n_edge][N_T]; C: device complex128 [n_edge][n_edge];
 *   V, X: device complex128 [nrhs][N_T + n_edge] (X: output; no initial guess).
 * The A-solves run ztoep_solve with opts (the n_edge solves for F in chunks of
 * up to 256 right-hand sides); info (host [nrhs], may be NULL) receives the
 * solves for U.  The contractions over N_T and n_edge are FP64; S is solved by
 * FP64 Gauss-Jordan elimination with partial pivoting.  Allocates
 * (n_edge + 2 nrhs) N_T + n_edge (n_edge + nrhs) complex128 of stream-ordered
 * workspace and returns after the work completes.  Errors: ARG, NOMEM, CUDA,
 * NONFINITE (singular S), and NOCONV/TIMEOUT from an A-solve (the solution is
 * still formed). */
ZTOEP_API ztoep_status_t ztoep_solve_schur(ztoep_plan_t plan_A, int32_t n_edge, const void *B, const void *C,
                                           const ztoep_solve_opts_t *opts, int32_t nrhs, const void *V, void *X,
                                           ztoep_solve_info_t *info, void *stream);

/* ---- Far field (Sec. III, Eqs. farfieldBasis and tensorProd) ----
 * Far field of the element currents on the array-factor grid of the plan's
 * embedding: direction f = ky*lx + kx has k a u = 2 pi kx / lx and
 * k a v = 2 pi ky / ly (u = sin th cos ph, v = sin th sin ph, a the element
 * period), so that the phase of part (m, n) at offset (m a, n a, 0) is
 * exp(2 pi j (kx m / lx + ky n / ly)).  With the per-basis far-field tensor
 * Fh of one element (Eq. farfieldBasis),
 *   F[r][f][t] = -j k eta sum_{active (m,n)} exp(j k r^_f . d_(m,n))
 *                sum_{i<b} I[r][(n*nx+m)*b+i] Fh[f][t][i]      (Eq. tensorProd),
 * computed as the plan's FP64 forward spectrum at -f and one b-term dot
 * product per (f, t, r).  Edge unknowns (other array components) are not
 * included.
 *   I: device complex128 [nrhs][N]; Fh: device complex128 [lx*ly][npol][b];
 *   F: device complex128 [nrhs][lx*ly][npol]; npol 1..16.
 * Stream-ordered; allocates F b nrhs complex128 of stream-ordered workspace.
 * Errors: ARG, NOMEM, CUDA. */
ZTOEP_API ztoep_status_t ztoep_far_field_grid(ztoep_plan_t plan, int32_t nrhs, const void *I, int32_t npol,
                                              const void *Fh, double k, double eta, void *F, void *stream);

/* Device bytes a plan for `desc` plus the workspace of a solve with up to
 * max_nrhs right-hand sides and restart length `restart` would use (for
 * admission control).  0 if the descriptor is invalid. */
ZTOEP_API size_t ztoep_footprint(const ztoep_desc_t *desc, int32_t max_nrhs, int32_t restart);

ZTOEP_API void ztoep_plan_destroy(ztoep_plan_t plan);

/* ---- Autotuning (not part of the method: launch and layout choices) ----
 * The choices a plan's kernels are built with.  0 in a field means the
 * built-in heuristic.  rad_order: 0 = radix 4 first, 1 = reversed sequence;
 * fft_channels: channels one CTA of an FP32 FFT pass transforms (1..64, a
 * power of two; 0 = heuristic), fft_threads: its block size (64/128/256) in
 * the shared-memory kernel; fft_kernel: 0 = heuristic (the register kernel
 * where the embedding size has one), 1 = shared-memory Stockham passes,
 * 2 = register passes (two small DFTs per point held in registers, one
 * shared-memory exchange; the shared-memory kernel where the size has none);
 * bp_split: threads per dot product of the SIMT block product (divides b);
 * tc_kchunk: complex K per CTA of the tensor-core B x_T product.  lx, ly,
 * rad_order, bp_split and tc_kchunk change the rounding of the products (all
 * choices compute the same product exactly in exact arithmetic); they are
 * fixed for the plan's life, so results stay independent of the batch. */
typedef struct {
    int32_t lx, ly;                   /* embedding sizes */
    int32_t rad_order_x, rad_order_y;
    int32_t fft_channels_x, fft_threads_x; /* FP32 x passes */
    int32_t fft_channels_y, fft_threads_y; /* FP32 y passes */
    int32_t fft_kernel_x, fft_kernel_y;    /* FP32 pass kernels (0, 1, 2) */
    int32_t bp_split, bp_ctas_per_sm; /* SIMT block product */
    int32_t tc_kchunk;                /* tensor-core edge product */
    int32_t nrhs;                     /* RHS count the choice was timed for */
    int32_t candidates;               /* configurations timed (0: taken from the cache) */
    double product_us;                /* FP32 product time with the choice */
    double default_us;                /* same with the heuristics and the smallest embedding */
} ztoep_tune_t;

/* Build a plan (same inputs and errors as ztoep_plan) whose embedding sizes,
 * FFT radix order, FFT-pass geometry, block-product split and tensor-core K
 * chunk minimise the measured FP32 product time for nrhs right-hand sides
 * (1..256).  Each candidate is timed with CUDA events on `stream`; embedding
 * candidates are the three smallest 5-smooth sizes >= 2N-1 per dimension
 * (within 25% of the smallest, unless desc fixes lx/ly) and each needs its
 * own plan build, so tuning costs several plan builds and about a hundred
 * products.  The choice is cached per (GPU name, nx, ny, b, n_edge, lx, ly
 * of desc, nrhs) in the process and, when the environment variable
 * ZTOEP_TUNE_CACHE names a file, in that file (one line per key), so a
 * later call builds the plan once with the cached choice.  tune (may be
 * NULL) receives the choice.  The device memory of two plans is needed while
 * tuning. */
ZTOEP_API ztoep_status_t ztoep_plan_autotune(const ztoep_desc_t *desc, const void *T, const void *B,
                                             const void *C, int32_t nrhs, void *stream, ztoep_plan_t *out,
                                             ztoep_tune_t *tune);

/* Build a plan with explicit choices (a ztoep_tune_t from ztoep_plan_autotune,
 * possibly of another process); desc's lx/ly are replaced by tune's when
 * nonzero.  ARG if a choice is out of range. */
ZTOEP_API ztoep_status_t ztoep_plan_tuned(const ztoep_desc_t *desc, const void *T, const void *B, const void *C,
                                          const ztoep_tune_t *tune, void *stream, ztoep_plan_t *out);

/* The choices of a plan (heuristic fields reported as 0). */
ZTOEP_API ztoep_status_t ztoep_plan_get_tune(ztoep_plan_t plan, ztoep_tune_t *tune);

ZTOEP_API const char *ztoep_status_string(ztoep_status_t status);

/* ---- Instrumentation (not part of the method) ----
 * Kernel classes: 0 FFT passes, 1 per-frequency block products, 2 edge
 * coupling (one pass over B), 3 Arnoldi/Givens steps, 4 everything else,
 * 5 tensor-core (tcgen05) complex GEMMs, lock-step kernel, 6 the same GEMMs,
 * warp-specialised pipelined kernel. */

/* Number of CUDA kernels this library has launched in this process. */
ZTOEP_API uint64_t ztoep_launch_count(void);

/* Time the launches of the classes whose bit is set in `mask` with a CUDA
 * event pair on the launching stream (0 = off, the default).  With
 * ZTOEP_TIMING_SERIAL also set, a product runs its edge branch on the
 * launching stream after the FFT chain instead of concurrently on its second
 * stream, so each timed kernel runs alone (graph captures are unaffected). */
#define ZTOEP_TIMING_SERIAL (1 << 30)
ZTOEP_API void ztoep_timing_enable(int32_t mask);

/* Forget accumulated timings (waits for pending events). */
ZTOEP_API void ztoep_timing_reset(void);

/* Timed launches of class `cls` since the last reset and their summed device
 * time in ms (waits for pending events).  Errors: ARG. */
ZTOEP_API ztoep_status_t ztoep_timing_read(int32_t cls, uint64_t *timed_launches, double *total_ms);

/* Library version string, e.g. "ztoep 0.1 sm_103a". */
ZTOEP_API const char *ztoep_version(void);

/* ---- Serving: continuous batching of array solves ----
 * A scheduler owns worker threads, each with its own CUDA stream.  Submitted
 * requests (any nx, ny, b, n_edge, nrhs) wait in a FIFO queue and are
 * admitted as soon as a worker is free and the device bytes they need fit in
 * the budget (ztoep_footprint of the request, plus, for host inputs, its
 * device staging copies of T, B and C, plus the plans kept resident);
 * admitted requests run concurrently, so their kernels overlap on the device.
 * Plans (the FFT'd generating blocks, B and C) stay resident under their
 * plan_key and are reused by later requests with the same key; idle ones are
 * evicted least-recently-used when the budget requires.  With group_max > 1
 * a worker takes the queue head together with the requests right behind it
 * that can share one grouped solve (ztoep_solve_group).  Each request gets
 * exactly the arithmetic of a ztoep_solve of the same request alone. */
typedef struct ztoep_sched_s *ztoep_sched_t;

typedef struct {
    size_t hbm_budget;   /* device bytes the scheduler may hold (plans + work) */
    int32_t workers;     /* concurrent requests (worker threads / streams), 1..64 */
    int32_t device;      /* CUDA device index */
    int32_t fake_backend;/* 1: no CUDA work; each request sleeps fake_us (host-logic tests) */
    int64_t fake_us;
    int32_t group_max;   /* up to this many queued requests (0..8; 0 and 1 = one at a time) that
                            follow each other in arrival order, have device inputs, equal options,
                            plans of their own and sizes within a factor 4 run as one
                            ztoep_solve_group; a group completes when its last member converges */
} ztoep_sched_opts_t;

typedef struct {
    ztoep_desc_t desc;
    int32_t inputs_on_device; /* 1: T, B, C, V and X are device pointers, else host */
    uint64_t plan_key;        /* nonzero: requests with equal keys share one resident plan */
    const void *T, *B, *C;    /* complex128, layouts as in ztoep_plan */
    int32_t nrhs;
    const void *V;            /* complex128 [nrhs][N] */
    void *X;                  /* complex128 [nrhs][N] solution (initial guess ignored) */
    ztoep_solve_opts_t opts;
    ztoep_solve_info_t *info; /* host [nrhs] or NULL */
} ztoep_request_t;
/* V and X must stay valid until the request completes; T, B and C until it
 * reports inputs_consumed (or completes). */

typedef struct {
    int32_t state;           /* 0 queued, 1 running, 2 done */
    int32_t status;          /* ztoep_status_t of the solve (when done) */
    int32_t plan_reused;     /* the resident plan of plan_key was used */
    int32_t inputs_consumed; /* 1 once the plan exists: T, B and C are no longer read */
    double queue_ms;         /* submit -> start */
    double latency_ms;       /* submit -> done */
} ztoep_request_state_t;

typedef struct {
    int64_t submitted, completed, max_in_flight;
    size_t bytes_in_use, peak_bytes, resident_plan_bytes;
    int64_t plans_built, plans_reused, plans_evicted;
    int64_t groups;      /* grouped solves run (two or more requests) */
} ztoep_sched_stats_t;

/* Errors: ARG (bad options), CUDA. */
ZTOEP_API ztoep_status_t ztoep_sched_create(const ztoep_sched_opts_t *opts, ztoep_sched_t *out);

/* Queue a request; *id identifies it.  A request whose footprint alone exceeds
 * the budget is rejected with NOMEM; a bad descriptor with ARG. */
ZTOEP_API ztoep_status_t ztoep_sched_submit(ztoep_sched_t s, const ztoep_request_t *req, int64_t *id);

/* Current state of request id (ARG if unknown). */
ZTOEP_API ztoep_status_t ztoep_sched_poll(ztoep_sched_t s, int64_t id, ztoep_request_state_t *st);

/* Block until request id is done or timeout_ms passes (TIMEOUT); < 0 waits forever. */
ZTOEP_API ztoep_status_t ztoep_sched_wait(ztoep_sched_t s, int64_t id, int64_t timeout_ms,
                                          ztoep_request_state_t *st);

ZTOEP_API ztoep_status_t ztoep_sched_get_stats(ztoep_sched_t s, ztoep_sched_stats_t *st);

/* Finish queued and running requests, free resident plans, stop the workers. */
ZTOEP_API void ztoep_sched_destroy(ztoep_sched_t s);

#ifdef __cplusplus
}
#endif

#endif /* ZTOEP_H */
