"""Python access to the CPU FP64 oracle (oracle.c) through ctypes.

TEST INFRASTRUCTURE ONLY: the slow, plain reference the GPU library is
checked against.  Only tests, the smoke check and the benchmark's CPU-baseline
leg use it.  It shares no code with the library; the only common module is
the seeded input generator (`paper_2506_04710_gb300.synth`).

Every function follows a plain definition from the paper:
  assemble      Z^part = [[A, B^T], [B, C]] (Eq. matrixForm) with A the
                two-level block Toeplitz matrix of Eq. submatrixAA,
                A[(m,n,i),(m',n',j)] = T[m-m', n-n'][i,j]; masked elements
                give identity rows/columns.
  matvec_*      y = Z x by direct summation (Eq. MoMMatrixEq's left side).
  lu_*          Z I = V by LU with partial pivoting.
  schur_solve   Eqs. solveEqSystem1/2 (Sec. II-D).
  assemble_points  Z[k,l] = G(|r_k - r_l|) + diag, from positions (Sec. II, G).
  gmres         restarted GMRES(m), FP64, matvec from the blocks (Sec. II-D).
  port_admittance, scattering
                the port matrices of Sec. IV-B: port currents from delta-port
                solutions, Y = L I^ L, Z_port = Y^-1, S by the power-wave
                definition (the paper's reference for S, its Eq. 18).
  far_field     Eq. tensorProd: F[m][t] = -j k eta sum_p sum_n
                exp(j k r^_m . d_p) I[n, p] F^[m][t][n] by direct summation.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)
import build as _build  # noqa: E402

_lib = None
c_i64 = ctypes.c_int64
c_int = ctypes.c_int
c_dbl = ctypes.c_double
c_p = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_assemble.argtypes = [c_int, c_int, c_int, c_int, c_p, c_p, c_p, c_p, c_p]
        L.oracle_matvec_dense.argtypes = [c_i64, c_p, c_int, c_p, c_p]
        L.oracle_matvec_blocks.argtypes = [c_int, c_int, c_int, c_int, c_p, c_p, c_p, c_p, c_int,
                                           c_p, c_p]
        L.oracle_matvec_rows.argtypes = [c_int, c_int, c_int, c_int, c_p, c_p, c_p, c_p, c_int,
                                         c_p, c_i64, c_p, c_p]
        L.oracle_assemble_points.argtypes = [c_i64, c_p, c_dbl, c_dbl, c_dbl, c_dbl, c_p, c_p]
        L.oracle_lu_factor.argtypes = [c_i64, c_p, c_p]
        L.oracle_lu_factor.restype = c_int
        L.oracle_lu_solve.argtypes = [c_i64, c_p, c_p, c_int, c_p]
        L.oracle_norm1.argtypes = [c_i64, c_p]
        L.oracle_norm1.restype = c_dbl
        L.oracle_inv_norm1_est.argtypes = [c_i64, c_p, c_p]
        L.oracle_inv_norm1_est.restype = c_dbl
        L.oracle_schur_solve.argtypes = [c_i64, c_i64, c_p, c_p, c_p, c_int, c_p, c_p]
        L.oracle_schur_solve.restype = c_int
        L.oracle_gmres.argtypes = [c_int, c_int, c_int, c_int, c_p, c_p, c_p, c_p, c_p, c_p, c_int,
                                   c_dbl, c_int, ctypes.POINTER(c_dbl)]
        L.oracle_gmres.restype = c_int
        _lib = L
    return _lib


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _prob_arrays(prob):
    T = _c(prob.T)
    B = _c(prob.B)
    C = _c(prob.C)
    act = _c(prob.active, np.uint8)
    return T, B, C, act


def assemble(prob) -> np.ndarray:
    T, B, C, act = _prob_arrays(prob)
    Z = np.empty((prob.n, prob.n), dtype=np.complex128)
    lib().oracle_assemble(prob.nx, prob.ny, prob.b, prob.n_edge, _ptr(T), _ptr(B), _ptr(C),
                          _ptr(act), _ptr(Z))
    return Z


def matvec_dense(Z: np.ndarray, X: np.ndarray) -> np.ndarray:
    Z = _c(Z)
    X = _c(np.atleast_2d(X))
    Y = np.empty_like(X)
    lib().oracle_matvec_dense(Z.shape[0], _ptr(Z), X.shape[0], _ptr(X), _ptr(Y))
    return Y


def matvec_blocks(prob, X: np.ndarray) -> np.ndarray:
    T, B, C, act = _prob_arrays(prob)
    X = _c(np.atleast_2d(X))
    Y = np.empty_like(X)
    lib().oracle_matvec_blocks(prob.nx, prob.ny, prob.b, prob.n_edge, _ptr(T), _ptr(B), _ptr(C),
                               _ptr(act), X.shape[0], _ptr(X), _ptr(Y))
    return Y


def matvec_rows(prob, X: np.ndarray, rows) -> np.ndarray:
    """(Z X[r])[rows] for each RHS r: [nrhs][len(rows)]."""
    T, B, C, act = _prob_arrays(prob)
    X = _c(np.atleast_2d(X))
    rows = _c(rows, np.int64)
    Y = np.empty((X.shape[0], rows.shape[0]), dtype=np.complex128)
    lib().oracle_matvec_rows(prob.nx, prob.ny, prob.b, prob.n_edge, _ptr(T), _ptr(B), _ptr(C),
                             _ptr(act), X.shape[0], _ptr(X), rows.shape[0], _ptr(rows), _ptr(Y))
    return Y


def assemble_points(pos: np.ndarray, k0: float, rmin: float, diag: complex,
                    unknown_mask: np.ndarray | None = None) -> np.ndarray:
    pos = _c(pos, np.float64)
    N = pos.shape[0]
    mask = None if unknown_mask is None else _c(unknown_mask, np.uint8)
    Z = np.empty((N, N), dtype=np.complex128)
    lib().oracle_assemble_points(N, _ptr(pos), k0, rmin, diag.real, diag.imag, _ptr(mask), _ptr(Z))
    return Z


class LU:
    """LU with partial pivoting of a dense matrix (oracle_lu_factor)."""

    def __init__(self, Z: np.ndarray):
        self.n = Z.shape[0]
        self.norm1 = lib().oracle_norm1(self.n, _ptr(_c(Z)))
        self.lu = np.array(Z, dtype=np.complex128, order="C", copy=True)
        self.piv = np.empty(self.n, dtype=np.int64)
        rc = lib().oracle_lu_factor(self.n, _ptr(self.lu), _ptr(self.piv))
        if rc != 0:
            raise np.linalg.LinAlgError(f"zero pivot in column {rc - 1}")

    def solve(self, V: np.ndarray) -> np.ndarray:
        X = np.array(np.atleast_2d(V), dtype=np.complex128, order="C", copy=True)
        lib().oracle_lu_solve(self.n, _ptr(self.lu), _ptr(self.piv), X.shape[0], _ptr(X))
        return X

    def cond1_estimate(self) -> float:
        """kappa_1 ~ ||Z||_1 * est(||Z^-1||_1) (Hager-Higham estimator)."""
        return self.norm1 * lib().oracle_inv_norm1_est(self.n, _ptr(self.lu), _ptr(self.piv))


def schur_solve(A: np.ndarray, B: np.ndarray, C: np.ndarray, V: np.ndarray) -> np.ndarray:
    A, B, C = _c(A), _c(B), _c(C)
    V = _c(np.atleast_2d(V))
    NT, E = A.shape[0], C.shape[0]
    X = np.empty_like(V)
    rc = lib().oracle_schur_solve(NT, E, _ptr(A), _ptr(B), _ptr(C), V.shape[0], _ptr(V), _ptr(X))
    if rc != 0:
        raise np.linalg.LinAlgError(f"schur solve failed ({rc})")
    return X


def gmres(prob, v: np.ndarray, x0: np.ndarray | None = None, restart: int = 30,
          tol: float = 1e-10, max_iter: int = 2000):
    """FP64 restarted GMRES on one RHS; returns (x, iterations, true relative residual)."""
    T, B, C, act = _prob_arrays(prob)
    v = _c(v)
    x = np.zeros(prob.n, np.complex128) if x0 is None else np.array(x0, np.complex128, copy=True)
    rel = c_dbl(0.0)
    it = lib().oracle_gmres(prob.nx, prob.ny, prob.b, prob.n_edge, _ptr(T), _ptr(B), _ptr(C),
                            _ptr(act), _ptr(v), _ptr(x), restart, tol, max_iter, ctypes.byref(rel))
    return x, it, rel.value


def unknown_mask(prob) -> np.ndarray:
    return np.concatenate([np.repeat(prob.active.reshape(-1), prob.b),
                           np.ones(prob.n_edge, np.uint8)]).astype(np.uint8)


def relres(prob_or_Z, X: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Per-RHS ||V - Z X|| / ||V||, matvec by the oracle."""
    if isinstance(prob_or_Z, np.ndarray):
        ZX = matvec_dense(prob_or_Z, X)
    else:
        ZX = matvec_blocks(prob_or_Z, X)
    V = np.atleast_2d(V)
    return np.linalg.norm(V - ZX, axis=1) / np.linalg.norm(V, axis=1)


def port_admittance(I: np.ndarray, ports, edge_len) -> np.ndarray:
    """Sec. IV-B.  With the excitation matrix V = [e_{i_1}, ..., e_{i_p}] the
    solution has one column per port; here I[k] (a row) is the solution for
    the delta excitation at port k.  The port currents I^[a][k] = I[k][i_a]
    (rows i_1..i_p of the current matrix), and Y = L I^ L with
    L = diag(1 / l_{i_1}, ..., 1 / l_{i_p}) (l: the ports' edge lengths)."""
    I = np.atleast_2d(np.asarray(I))
    ports = np.asarray(ports, dtype=np.int64)
    Ihat = I[:, ports].T
    L = np.diag(1.0 / np.asarray(edge_len, dtype=np.float64))
    return L @ Ihat @ L


def scattering(Y: np.ndarray, z0) -> np.ndarray:
    """Sec. IV-B: the port impedance matrix Z_port = Y^-1 and, with the
    reference impedances z0, the power-wave scattering matrix
    S = F (Z_port - G*) (Z_port + G)^-1 F^-1, G = diag(z0),
    F = diag(1 / (2 sqrt(|Re z0|)))."""
    Zp = np.linalg.inv(np.asarray(Y, dtype=np.complex128))
    z0 = np.asarray(z0, dtype=np.complex128)
    G = np.diag(z0)
    F = np.diag(1.0 / (2.0 * np.sqrt(np.abs(z0.real))))
    return F @ (Zp - G.conj()) @ np.linalg.inv(Zp + G) @ np.linalg.inv(F)


def far_field(prob, I: np.ndarray, uv: np.ndarray, Fh: np.ndarray, k: float, eta: float) -> np.ndarray:
    """Eq. tensorProd for the element component: parts p = active elements
    (m, n) at offsets d_p = (m a, n a, 0), basis coefficients I[r][(n nx + m) b + i],
    F^ = Fh[M][T][b] (Eq. farfieldBasis), directions (u, v) = (sin th cos ph,
    sin th sin ph) so that k r^.d_p = k a (u m + v n):
        F[r][m][t] = -j k eta sum_p exp(j k r^_m.d_p) sum_i I[r][p b + i] Fh[m][t][i].
    Direct summation over the parts, no FFT.  Returns [nrhs][M][T]."""
    from paper_2506_04710_gb300.synth import PERIOD
    I = np.atleast_2d(np.asarray(I))
    uv = np.asarray(uv, dtype=np.float64)
    out = np.zeros((I.shape[0], len(uv), Fh.shape[1]), np.complex128)
    b = prob.b
    for n in range(prob.ny):
        for m in range(prob.nx):
            if not prob.active[n, m]:
                continue
            p = n * prob.nx + m
            ph = np.exp(1j * k * PERIOD * (uv[:, 0] * m + uv[:, 1] * n))  # [M]
            Ip = I[:, p * b:(p + 1) * b]                                   # [r][b]
            out += ph[None, :, None] * np.einsum("mti,ri->rmt", Fh, Ip)
    return -1j * k * eta * out
