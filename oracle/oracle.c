/*
 * CPU FP64 oracle for the two-level block-Toeplitz array system.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * GPU library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the library never does.  It
 * shares no code, header or table with the GPU path.
 *
 * Everything is complex double, interleaved (re, im), row-major.
 *
 * Definitions followed (paper sections / equations):
 *  - Z I = V, the MoM matrix equation (Sec. II, Eq. MoMMatrixEq).
 *  - Z^part = [[A, B^T], [B, C]] (Sec. II-C, Eq. matrixForm): A couples the
 *    element parts, B the margin (edge) parts to the element parts, C the
 *    margin parts among themselves.  The B^T block follows from the symmetry
 *    of Z (Sec. II-A).
 *  - A is two-level block Toeplitz (Eq. submatrixAA): outer level over the
 *    element row n (y), inner level over the element column m (x), x fastest
 *    (part indexing of Sec. II-C).  Its block at element pair
 *    ((m,n),(m',n')) is the generating block T[m-m', n-n'].
 *  - Inactive (masked) elements: Z' = M Z M + (I - M), M = diag(mask).
 *  - Schur-complement solve (Sec. II-D, Eqs. solveEqSystem1/2).
 *
 * Array conventions shared with the generator (not with the GPU code):
 *   T: [2ny-1][2nx-1][b][b], T[q+ny-1][p+nx-1] = block for offset (p, q).
 *   B: [E][NT], C: [E][E], active: [ny][nx], X/Y/V: [nrhs][N].
 *   Unknown (m, n, i) -> (n*nx + m)*b + i; edge unknown e -> NT + e.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static inline int64_t toep_index(int nx, int b, int m, int n, int i) {
    return ((int64_t)n * nx + m) * b + i;
}

static inline int unknown_active(int nx, int ny, int b, const uint8_t *active, int64_t k) {
    int64_t nt = (int64_t)nx * ny * b;
    if (k >= nt || active == NULL) return 1;
    return active[k / b] != 0;
}

/* Entry Z[k][l] of the unmasked matrix, straight from the definition. */
static cplx entry_unmasked(int nx, int ny, int b, int E, const cplx *T, const cplx *B,
                           const cplx *C, int64_t k, int64_t l) {
    int64_t nt = (int64_t)nx * ny * b;
    if (k < nt && l < nt) {
        int64_t ek = k / b, el = l / b;
        int i = (int)(k % b), j = (int)(l % b);
        int m = (int)(ek % nx), n = (int)(ek / nx);
        int m2 = (int)(el % nx), n2 = (int)(el / nx);
        int p = m - m2, q = n - n2;
        const cplx *blk = T + (((int64_t)(q + ny - 1) * (2 * nx - 1) + (p + nx - 1)) * b) * b;
        return blk[(int64_t)i * b + j];
    }
    if (k >= nt && l < nt) return B[(k - nt) * nt + l];
    if (k < nt && l >= nt) return B[(l - nt) * nt + k];
    return C[(k - nt) * E + (l - nt)];
}

static cplx entry(int nx, int ny, int b, int E, const cplx *T, const cplx *B, const cplx *C,
                  const uint8_t *active, int64_t k, int64_t l) {
    int ak = unknown_active(nx, ny, b, active, k), al = unknown_active(nx, ny, b, active, l);
    if (ak && al) return entry_unmasked(nx, ny, b, E, T, B, C, k, l);
    return (k == l) ? 1.0 : 0.0;
}

/* Dense Z [N][N] (N = nx*ny*b + E). */
void oracle_assemble(int nx, int ny, int b, int E, const cplx *T, const cplx *B, const cplx *C,
                     const uint8_t *active, cplx *Z) {
    int64_t N = (int64_t)nx * ny * b + E;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k)
        for (int64_t l = 0; l < N; ++l)
            Z[k * N + l] = entry(nx, ny, b, E, T, B, C, active, k, l);
}

/* Y[r] = Z X[r], direct O(N^2) sum per row. */
void oracle_matvec_dense(int64_t N, const cplx *Z, int nrhs, const cplx *X, cplx *Y) {
#pragma omp parallel for collapse(2) schedule(static)
    for (int r = 0; r < nrhs; ++r)
        for (int64_t k = 0; k < N; ++k) {
            cplx s = 0;
            const cplx *x = X + (int64_t)r * N;
            const cplx *z = Z + k * N;
            for (int64_t l = 0; l < N; ++l) s += z[l] * x[l];
            Y[(int64_t)r * N + k] = s;
        }
}

/* Y = Z X without forming Z: each entry is read from the generating blocks on
 * the fly (same definition as oracle_assemble).  For systems whose dense Z
 * does not fit in host memory. */
void oracle_matvec_blocks(int nx, int ny, int b, int E, const cplx *T, const cplx *B,
                          const cplx *C, const uint8_t *active, int nrhs, const cplx *X,
                          cplx *Y) {
    int64_t N = (int64_t)nx * ny * b + E;
#pragma omp parallel for collapse(2) schedule(dynamic, 16)
    for (int r = 0; r < nrhs; ++r)
        for (int64_t k = 0; k < N; ++k) {
            const cplx *x = X + (int64_t)r * N;
            cplx s = 0;
            for (int64_t l = 0; l < N; ++l)
                s += entry(nx, ny, b, E, T, B, C, active, k, l) * x[l];
            Y[(int64_t)r * N + k] = s;
        }
}

/* Same as oracle_matvec_blocks for a subset of output rows: Y[r][s] = (Z X[r])[rows[s]]. */
void oracle_matvec_rows(int nx, int ny, int b, int E, const cplx *T, const cplx *B,
                        const cplx *C, const uint8_t *active, int nrhs, const cplx *X,
                        int64_t nrows, const int64_t *rows, cplx *Y) {
    int64_t N = (int64_t)nx * ny * b + E;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int r = 0; r < nrhs; ++r)
        for (int64_t s = 0; s < nrows; ++s) {
            const cplx *x = X + (int64_t)r * N;
            int64_t k = rows[s];
            cplx acc = 0;
            for (int64_t l = 0; l < N; ++l)
                acc += entry(nx, ny, b, E, T, B, C, active, k, l) * x[l];
            Y[(int64_t)r * nrows + s] = acc;
        }
}

/* Regularised free-space Green's function exp(-jkR')/(4 pi R'), R' = max(R, rmin)
 * (Sec. II, G(r, r') = exp(-jk|r-r'|)/(4 pi |r-r'|)). */
static cplx green(double R, double k0, double rmin) {
    double Rp = R > rmin ? R : rmin;
    return cexp(-I * k0 * Rp) / (4.0 * M_PI * Rp);
}

/* Z straight from the unknowns' positions [N][2] (z = 0): Z[k][l] = G(|r_k - r_l|)
 * + diag on k == l, then the activity mask.  Independent of the block layout;
 * used to check the Toeplitz assembly against the physics it encodes. */
void oracle_assemble_points(int64_t N, const double *pos, double k0, double rmin, double diag_re,
                            double diag_im, const uint8_t *unknown_mask, cplx *Z) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < N; ++k)
        for (int64_t l = 0; l < N; ++l) {
            int ak = unknown_mask ? unknown_mask[k] : 1, al = unknown_mask ? unknown_mask[l] : 1;
            cplx z;
            if (ak && al) {
                double dx = pos[2 * k] - pos[2 * l], dy = pos[2 * k + 1] - pos[2 * l + 1];
                z = green(sqrt(dx * dx + dy * dy), k0, rmin);
                if (k == l) z += diag_re + I * diag_im;
            } else {
                z = (k == l) ? 1.0 : 0.0;
            }
            Z[k * N + l] = z;
        }
}

/* LU factorisation with partial pivoting, in place (PA = LU, unit lower L).
 * Right-looking textbook elimination (Golub & Van Loan, Alg. 3.4.1).
 * Returns 0, or k+1 if the pivot of column k is exactly zero. */
int oracle_lu_factor(int64_t N, cplx *A, int64_t *piv) {
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = k;
        double best = cabs(A[k * N + k]);
        for (int64_t i = k + 1; i < N; ++i) {
            double v = cabs(A[i * N + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return (int)(k + 1);
        if (p != k)
            for (int64_t j = 0; j < N; ++j) {
                cplx t = A[k * N + j]; A[k * N + j] = A[p * N + j]; A[p * N + j] = t;
            }
        cplx inv = 1.0 / A[k * N + k];
#pragma omp parallel for schedule(static)
        for (int64_t i = k + 1; i < N; ++i) {
            cplx l = A[i * N + k] * inv;
            A[i * N + k] = l;
            double lr = creal(l), li = cimag(l);
            double *ai = (double *)(A + i * N);
            const double *ak = (const double *)(A + k * N);
            for (int64_t j = k + 1; j < N; ++j) {
                double ur = ak[2 * j], ui = ak[2 * j + 1];
                ai[2 * j] -= lr * ur - li * ui;
                ai[2 * j + 1] -= lr * ui + li * ur;
            }
        }
    }
    return 0;
}

/* Solve (PA) X = V in place using the factors of oracle_lu_factor. X: [nrhs][N]. */
void oracle_lu_solve(int64_t N, const cplx *LU, const int64_t *piv, int nrhs, cplx *X) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < nrhs; ++r) {
        cplx *x = X + (int64_t)r * N;
        for (int64_t k = 0; k < N; ++k)
            if (piv[k] != k) { cplx t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
        for (int64_t i = 0; i < N; ++i) {
            cplx s = x[i];
            for (int64_t j = 0; j < i; ++j) s -= LU[i * N + j] * x[j];
            x[i] = s;
        }
        for (int64_t i = N - 1; i >= 0; --i) {
            cplx s = x[i];
            for (int64_t j = i + 1; j < N; ++j) s -= LU[i * N + j] * x[j];
            x[i] = s / LU[i * N + i];
        }
    }
}

/* 1-norm of a dense matrix: max column sum of |a_ij|. */
double oracle_norm1(int64_t N, const cplx *A) {
    double best = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        double s = 0.0;
        for (int64_t i = 0; i < N; ++i) s += cabs(A[i * N + j]);
        if (s > best) best = s;
    }
    return best;
}

/* Solve (PA)^H x = y with the LU factors: A^H = U^H L^H P. */
static void lu_solve_herm(int64_t N, const cplx *LU, const int64_t *piv, cplx *x) {
    for (int64_t i = 0; i < N; ++i) { /* U^H z = y (lower triangular) */
        cplx s = x[i];
        for (int64_t j = 0; j < i; ++j) s -= conj(LU[j * N + i]) * x[j];
        x[i] = s / conj(LU[i * N + i]);
    }
    for (int64_t i = N - 1; i >= 0; --i) { /* L^H w = z (unit upper) */
        cplx s = x[i];
        for (int64_t j = i + 1; j < N; ++j) s -= conj(LU[j * N + i]) * x[j];
        x[i] = s;
    }
    for (int64_t k = N - 1; k >= 0; --k) /* x = P^T w */
        if (piv[k] != k) { cplx t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
}

/* Estimate of ||A^-1||_1 by Hager's method as refined by Higham
 * (Hager, SIAM J. Sci. Stat. Comput. 5, 1984; Higham, ACM TOMS 14, 1988,
 * complex version with sign(z) = z/|z|).  Uses the LU factors. */
double oracle_inv_norm1_est(int64_t N, const cplx *LU, const int64_t *piv) {
    cplx *x = malloc(sizeof(cplx) * N);
    double est = 0.0;
    for (int64_t i = 0; i < N; ++i) x[i] = 1.0 / (double)N;
    for (int it = 0; it < 5; ++it) {
        oracle_lu_solve(N, LU, piv, 1, x); /* x = A^-1 x */
        double g = 0.0;
        for (int64_t i = 0; i < N; ++i) g += cabs(x[i]);
        if (it > 0 && g <= est) { est = g > est ? g : est; break; }
        est = g;
        for (int64_t i = 0; i < N; ++i) {
            double a = cabs(x[i]);
            x[i] = a > 0 ? x[i] / a : 1.0;
        }
        lu_solve_herm(N, LU, piv, x); /* z = A^-H sign(x) */
        int64_t jmax = 0;
        double zmax = -1.0;
        for (int64_t i = 0; i < N; ++i) {
            double a = cabs(x[i]);
            if (a > zmax) { zmax = a; jmax = i; }
        }
        for (int64_t i = 0; i < N; ++i) x[i] = 0.0;
        x[jmax] = 1.0;
    }
    /* Higham's alternative lower bound with the alternating-sign vector. */
    for (int64_t i = 0; i < N; ++i)
        x[i] = ((i % 2) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(N > 1 ? N - 1 : 1));
    oracle_lu_solve(N, LU, piv, 1, x);
    double alt = 0.0;
    for (int64_t i = 0; i < N; ++i) alt += cabs(x[i]);
    alt = 2.0 * alt / (3.0 * (double)N);
    free(x);
    return alt > est ? alt : est;
}

/* Schur-complement solve of [[A, B^T], [B, C]] I = [V1; V2] (Sec. II-D):
 *   A [U F] = [V1  B^T],   I2 = (C - B F)^-1 (V2 - B U),   I1 = U - F I2.
 * With V2 = 0 this is the paper's I2 = -(C - BF)^-1 B U.  A (NT x NT), B
 * (E x NT), C (E x E) are dense; V is [nrhs][NT+E]; X receives the solution.
 * Both inner systems are solved with oracle_lu_factor/solve.  Returns 0 on
 * success. */
int oracle_schur_solve(int64_t NT, int64_t E, const cplx *A, const cplx *B, const cplx *C,
                       int nrhs, const cplx *V, cplx *X) {
    int64_t N = NT + E;
    cplx *LA = malloc(sizeof(cplx) * NT * NT);
    int64_t *pa = malloc(sizeof(int64_t) * NT);
    cplx *F = malloc(sizeof(cplx) * E * NT);   /* columns of F stored as rows: F^T [E][NT] */
    cplx *U = malloc(sizeof(cplx) * nrhs * NT); /* [nrhs][NT] */
    cplx *S = malloc(sizeof(cplx) * E * E);
    int64_t *ps = malloc(sizeof(int64_t) * (E > 0 ? E : 1));
    cplx *R = malloc(sizeof(cplx) * nrhs * (E > 0 ? E : 1));
    int rc = 0;
    memcpy(LA, A, sizeof(cplx) * NT * NT);
    if ((rc = oracle_lu_factor(NT, LA, pa)) != 0) goto out;
    /* F: column e of F solves A f = (B^T)[:, e] = B[e, :]. */
    memcpy(F, B, sizeof(cplx) * E * NT);
    oracle_lu_solve(NT, LA, pa, (int)E, F);
    for (int r = 0; r < nrhs; ++r) memcpy(U + r * NT, V + (int64_t)r * N, sizeof(cplx) * NT);
    oracle_lu_solve(NT, LA, pa, nrhs, U);
    if (E > 0) {
        /* S = C - B F, S[e][e2] = C[e][e2] - sum_t B[e][t] F[t][e2]. */
        for (int64_t e = 0; e < E; ++e)
            for (int64_t e2 = 0; e2 < E; ++e2) {
                cplx s = C[e * E + e2];
                for (int64_t t = 0; t < NT; ++t) s -= B[e * NT + t] * F[e2 * NT + t];
                S[e * E + e2] = s;
            }
        /* R = V2 - B U */
        for (int r = 0; r < nrhs; ++r)
            for (int64_t e = 0; e < E; ++e) {
                cplx s = V[(int64_t)r * N + NT + e];
                for (int64_t t = 0; t < NT; ++t) s -= B[e * NT + t] * U[r * NT + t];
                R[r * E + e] = s;
            }
        if ((rc = oracle_lu_factor(E, S, ps)) != 0) { rc += 1000000; goto out; }
        oracle_lu_solve(E, S, ps, nrhs, R); /* R <- I2 */
    }
    for (int r = 0; r < nrhs; ++r) {
        for (int64_t t = 0; t < NT; ++t) {
            cplx s = U[r * NT + t];
            for (int64_t e = 0; e < E; ++e) s -= F[e * NT + t] * R[r * E + e];
            X[(int64_t)r * N + t] = s;
        }
        for (int64_t e = 0; e < E; ++e) X[(int64_t)r * N + NT + e] = R[r * E + e];
    }
out:
    free(LA); free(pa); free(F); free(U); free(S); free(ps); free(R);
    return rc;
}

/* Restarted GMRES(m) in FP64 with modified Gram-Schmidt Arnoldi and Givens
 * rotations (Saad & Schultz, SIAM J. Sci. Stat. Comput. 7, 1986), matvec by
 * oracle_matvec_blocks.  One RHS v [N]; x [N] is the initial guess on entry
 * and the iterate on exit.  Stops when ||v - Z x|| <= tol ||v|| (true
 * residual checked at each restart) or after max_iter iterations.  Returns the
 * number of iterations; *relres receives the final true relative residual. */
int oracle_gmres(int nx, int ny, int b, int E, const cplx *T, const cplx *B, const cplx *C,
                 const uint8_t *active, const cplx *v, cplx *x, int m, double tol, int max_iter,
                 double *relres) {
    int64_t N = (int64_t)nx * ny * b + E;
    cplx *Vb = malloc(sizeof(cplx) * (m + 1) * N);
    cplx *H = calloc((size_t)(m + 1) * m, sizeof(cplx));
    cplx *g = malloc(sizeof(cplx) * (m + 1));
    cplx *cs = malloc(sizeof(cplx) * m), *sn = malloc(sizeof(cplx) * m);
    cplx *y = malloc(sizeof(cplx) * m);
    cplx *w = malloc(sizeof(cplx) * N);
    double vnorm = 0.0;
    for (int64_t k = 0; k < N; ++k) vnorm += creal(v[k] * conj(v[k]));
    vnorm = sqrt(vnorm);
    int iters = 0;
    double rel = 1.0;
    for (;;) {
        oracle_matvec_blocks(nx, ny, b, E, T, B, C, active, 1, x, w);
        double beta = 0.0;
        for (int64_t k = 0; k < N; ++k) { w[k] = v[k] - w[k]; beta += creal(w[k] * conj(w[k])); }
        beta = sqrt(beta);
        rel = vnorm > 0 ? beta / vnorm : 0.0;
        if (rel <= tol || iters >= max_iter || beta == 0.0) break;
        for (int64_t k = 0; k < N; ++k) Vb[k] = w[k] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0;
        g[0] = beta;
        int j;
        for (j = 0; j < m && iters < max_iter; ++j, ++iters) {
            oracle_matvec_blocks(nx, ny, b, E, T, B, C, active, 1, Vb + j * N, w);
            for (int i = 0; i <= j; ++i) {
                cplx h = 0;
                for (int64_t k = 0; k < N; ++k) h += conj(Vb[i * N + k]) * w[k];
                H[i * m + j] = h;
                for (int64_t k = 0; k < N; ++k) w[k] -= h * Vb[i * N + k];
            }
            double hn = 0.0;
            for (int64_t k = 0; k < N; ++k) hn += creal(w[k] * conj(w[k]));
            hn = sqrt(hn);
            H[(j + 1) * m + j] = hn;
            if (hn > 0)
                for (int64_t k = 0; k < N; ++k) Vb[(j + 1) * N + k] = w[k] / hn;
            for (int i = 0; i < j; ++i) { /* apply old rotations */
                cplx a = H[i * m + j], c = H[(i + 1) * m + j];
                H[i * m + j] = conj(cs[i]) * a + conj(sn[i]) * c;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
            }
            cplx a = H[j * m + j], c = H[(j + 1) * m + j];
            double d = sqrt(creal(a * conj(a)) + creal(c * conj(c)));
            cs[j] = d > 0 ? a / d : 1.0;
            sn[j] = d > 0 ? c / d : 0.0;
            H[j * m + j] = d;
            H[(j + 1) * m + j] = 0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = conj(cs[j]) * g[j];
            if (cabs(g[j + 1]) <= tol * vnorm) { ++j; ++iters; break; }
        }
        for (int i = j - 1; i >= 0; --i) { /* back substitution */
            cplx s = g[i];
            for (int l = i + 1; l < j; ++l) s -= H[i * m + l] * y[l];
            y[i] = s / H[i * m + i];
        }
        for (int i = 0; i < j; ++i)
            for (int64_t k = 0; k < N; ++k) x[k] += y[i] * Vb[i * N + k];
    }
    *relres = rel;
    free(Vb); free(H); free(g); free(cs); free(sn); free(y); free(w);
    return iters;
}
