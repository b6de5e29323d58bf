"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each check ties one part of the oracle (or of the seeded generator whose
arrays both sides consume) to something independent: the physics the blocks
encode (assembly straight from the unknowns' positions), closed forms,
published generator outputs, library routines that implement the textbook
definition (LAPACK solve, 2-D convolution, FFT), the paper's own counting
formulas and quoted memory sizes, and brute force on tiny inputs.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.signal

import oracle
from paper_2506_04710_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_problems():
    return [
        synth.make_problem(4, 4, 8, 16, seed=0),                      # the 4x4, b=8 workload
        synth.make_problem(3, 5, 4, 12, seed=7, rhs="planewave", nrhs=3),
        synth.make_problem(5, 3, 3, 10, seed=3, gap_column=2, edge_layout="split", rhs="ports"),
        synth.make_problem(1, 1, 6, 5, seed=11),
        synth.make_problem(2, 3, 1, 0, seed=5),
    ]


# ---------------------------------------------------------------- generator

def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLDEN, "splitmix64_seed1234567.json")))
    with np.errstate(over="ignore"):
        k = np.arange(1, 6, dtype=np.uint64)
        z = synth._mix64(np.uint64(g["seed"]) + k * synth.GAMMA)
    assert [int(v) for v in z] == [int(s) for s in g["first_outputs_u64"]]
    # uniform() is the top 53 bits of the same stream (stream 0, offset 0)
    u = synth.uniform(g["seed"], 0, 5)
    assert np.array_equal(u, (z >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)


def test_uniform_counter_based_offsets():
    a = synth.uniform(42, 1, 100)
    b = synth.uniform(42, 1, 60, offset=40)
    assert np.array_equal(a[40:], b)
    assert (a >= 0).all() and (a < 1).all()
    assert not np.array_equal(a, synth.uniform(42, 2, 100))


def test_green_closed_forms():
    # G(R) = exp(-jkR)/(4 pi R), k = 2 pi: R = 1/2 -> -1/(2 pi); R = 1/4 -> -j/pi.
    assert abs(synth.green_reg(np.array(0.5)) - (-1 / (2 * math.pi))) < 1e-16
    assert abs(synth.green_reg(np.array(0.25)) - (-1j / math.pi)) < 1e-16
    # regularised self term: R' = 0.05
    g0 = np.exp(-1j * 0.1 * math.pi) / (0.2 * math.pi)
    assert abs(synth.green_reg(np.array(0.0)) - g0) < 1e-15
    # the oracle's own Green's function (assemble_points) agrees
    pos = np.array([[0.0, 0.0], [0.3, 0.4]])  # |d| = 0.5
    Z = oracle.assemble_points(pos, synth.K0, synth.R_MIN, synth.DIAG)
    assert abs(Z[0, 1] - (-1 / (2 * math.pi))) < 1e-15
    assert abs(Z[0, 0] - (g0 + synth.DIAG)) < 1e-15


def test_blocks_transpose_symmetry_bitwise():
    # Z = Z^T (Sec. II-A) => T[-p,-q] = T[p,q]^T; the generator forms dx so this is exact.
    for prob in small_problems():
        T = prob.T
        assert np.array_equal(T[::-1, ::-1], np.transpose(T, (0, 1, 3, 2)))


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (4, 6), (5, 5), (7, 2)])
def test_unique_block_count_matches_paper(nx, ny):
    # Sec. II-C: A needs NxNy + (Nx-1)(Ny-1) submatrix calculations once both
    # Toeplitz levels and the symmetry are used; Eq. calcScalingA gives
    # (2NxNy - Nx - Ny + 1) e5^2 entries.
    b = 3
    pts = synth.basis_points(nx * 100 + ny, b)
    T = synth.toeplitz_blocks(pts, nx, ny)
    seen = set()
    for blk in T.reshape(-1, b, b):
        key = min(blk.tobytes(), blk.T.copy().tobytes())
        seen.add(key)
    assert len(seen) == nx * ny + (nx - 1) * (ny - 1)
    assert len(seen) * b * b == (2 * nx * ny - nx - ny + 1) * b * b


def test_paper_dense_memory_figures():
    # Sec. III-B/III-C quote the dense sizes of the directly meshed arrays;
    # N^2 entries of 16 bytes reproduce them, fixing complex128 as the
    # paper's entry size (and the oracle's precision).
    g = json.load(open(os.path.join(GOLDEN, "paper_memory.json")))
    for case in g["cases"]:
        nbytes = case["edges"] ** 2 * 16
        scale = {"GB": 1e9, "TB": 1e12}[case["unit"]]
        assert float(f"{nbytes / scale:.{case['digits']}g}") == pytest.approx(case["quoted"])


def test_memory_formula_reduces_as_paper_states():
    # Appendix Eqs. calcScalingA/B/C with e2=e8=e6=e4=e_m, e3=e9=e1=e7=e_c,
    # e5=e_E reduce to Eq. calcScalingApproxNew, reading its "4_Ny" as 4 N_y.
    sympy = pytest.importorskip("sympy")
    Nx, Ny, eE, em, ec = sympy.symbols("Nx Ny eE em ec")
    e = {1: ec, 3: ec, 7: ec, 9: ec, 2: em, 4: em, 6: em, 8: em, 5: eE}
    memA = (2 * Nx * Ny - Nx - Ny + 1) * e[5] ** 2
    memB = ((2 * Nx * Ny - Nx) * e[5] * (e[2] + e[8]) + (2 * Nx * Ny - Ny) * e[5] * (e[6] + e[4])
            + Nx * Ny * e[5] * (e[3] + e[9] + e[1] + e[7]))
    s4 = e[3] + e[9] + e[1] + e[7]
    memC = (Nx * Ny * (e[2] + e[8]) * (e[4] + e[6]) + Ny * (e[2] ** 2 + e[8] ** 2)
            + Nx * (e[6] ** 2 + e[4] ** 2) + (2 * Ny - 1) * e[2] * e[8] + (2 * Nx - 1) * e[6] * e[4]
            + (Nx * (e[6] + e[4]) + Ny * (e[2] + e[8])) * s4 + e[7] ** 2
            + e[3] * s4 + e[9] * (e[9] + e[1] + e[7]) + e[1] * (e[1] + e[7]))
    approx = ((2 * Nx * Ny - Nx - Ny + 1) * eE ** 2 + (8 * Nx * Ny - 2 * Nx - 2 * Ny) * eE * em
              + 4 * Nx * Ny * eE * ec + (4 * Nx * Ny + 4 * Nx + 4 * Ny - 2) * em ** 2
              + 8 * (Nx + Ny) * em * ec + 10 * ec ** 2)
    assert sympy.expand(memA + memB + memC - approx) == 0


# ---------------------------------------------------------------- assembly

def test_assembly_matches_physics_from_points():
    # The Toeplitz assembly (Eq. submatrixAA + Eq. matrixForm) must reproduce
    # Z[k,l] = G(|r_k - r_l|) (+ diag) evaluated directly between the unknowns'
    # positions, masked as M Z M + (I - M).  Not bitwise: dx is rounded in a
    # different order.
    for prob in small_problems():
        Z = oracle.assemble(prob)
        Zp = oracle.assemble_points(synth.unknown_positions(prob), synth.K0, synth.R_MIN,
                                    synth.DIAG, oracle.unknown_mask(prob))
        assert np.max(np.abs(Z - Zp)) <= 1e-13 * np.max(np.abs(Zp)), prob.name


def test_assembly_pin_catches_planted_mistakes():
    # Planted in oracle inputs on the CPU: a transposed generating block set
    # and a flipped offset sign must both fail the physics pin.
    prob = synth.make_problem(3, 4, 4, 8, seed=2)
    Zp = oracle.assemble_points(synth.unknown_positions(prob), synth.K0, synth.R_MIN, synth.DIAG)
    import copy
    bad1 = copy.copy(prob)
    bad1.T = np.ascontiguousarray(np.transpose(prob.T, (0, 1, 3, 2)))
    bad2 = copy.copy(prob)
    bad2.T = np.ascontiguousarray(prob.T[:, ::-1])
    for bad in (bad1, bad2):
        Z = oracle.assemble(bad)
        assert np.max(np.abs(Z - Zp)) > 1e-3


def test_assembly_symmetric_bitwise():
    for prob in small_problems():
        Z = oracle.assemble(prob)
        assert np.array_equal(Z, Z.T)


def test_single_element_is_plain_block_matrix():
    prob = synth.make_problem(1, 1, 6, 5, seed=11)
    Z = oracle.assemble(prob)
    ref = np.block([[prob.T[0, 0], prob.B.T], [prob.B, prob.C]])
    assert np.array_equal(Z, ref)


def test_scalar_two_level_toeplitz_is_2d_convolution():
    # b = 1, E = 0: y[n,m] = sum T[m-m', n-n'] x[n',m'] is a 2-D linear
    # convolution; scipy.signal.convolve2d is the textbook definition.
    for nx, ny in [(3, 4), (5, 2), (1, 6)]:
        prob = synth.make_problem(nx, ny, 1, 0, seed=nx * 10 + ny, rhs="planewave", nrhs=2)
        K = prob.T[:, :, 0, 0]  # K[q+ny-1, p+nx-1]
        Y = oracle.matvec_dense(oracle.assemble(prob), prob.V)
        for r in range(2):
            x = prob.V[r].reshape(ny, nx)
            full = scipy.signal.convolve2d(x, K, mode="full")
            ref = full[ny - 1:2 * ny - 1, nx - 1:2 * nx - 1]
            assert np.allclose(Y[r].reshape(ny, nx), ref, rtol=1e-13, atol=1e-13)


def fft_embedded_matvec(prob, X, Lx, Ly):
    """Circulant embedding + 2-D FFT over (m, n) + per-frequency block product
    + inverse FFT + crop, written with numpy.fft for this check only."""
    nx, ny, b, nt = prob.nx, prob.ny, prob.b, prob.n_toep
    emb = np.zeros((Ly, Lx, b, b), complex)
    for q in range(-(ny - 1), ny):
        for p in range(-(nx - 1), nx):
            emb[q % Ly, p % Lx] = prob.T[q + ny - 1, p + nx - 1]
    That = np.fft.fft2(emb, axes=(0, 1))
    mask_t = np.repeat(prob.active.reshape(-1), b).astype(float)
    out = np.empty_like(X)
    for r in range(X.shape[0]):
        xt = X[r, :nt] * mask_t
        xe = X[r, nt:]
        pad = np.zeros((Ly, Lx, b), complex)
        pad[:ny, :nx] = xt.reshape(ny, nx, b)
        Yh = np.einsum("yxij,yxj->yxi", That, np.fft.fft2(pad, axes=(0, 1)))
        yt = np.fft.ifft2(Yh, axes=(0, 1))[:ny, :nx].reshape(-1)
        yt = yt + prob.B.T @ xe
        yt = yt * mask_t + (1 - mask_t) * X[r, :nt]
        ye = prob.B @ xt + prob.C @ xe
        out[r] = np.concatenate([yt, ye])
    return out


@pytest.mark.parametrize("nx,ny,b,E", [(1, 1, 2, 0), (2, 3, 3, 4), (4, 2, 4, 6), (5, 5, 2, 8),
                                       (3, 4, 4, 0)])
def test_circulant_embedded_product_equals_dense(nx, ny, b, E):
    prob = synth.make_problem(nx, ny, b, E, seed=b, rhs="planewave", nrhs=2)
    Yd = oracle.matvec_dense(oracle.assemble(prob), prob.V)
    for Lx in range(2 * nx - 1, 2 * nx + 4):
        for Ly in range(2 * ny - 1, 2 * ny + 4):
            Yf = fft_embedded_matvec(prob, prob.V, Lx, Ly)
            assert np.max(np.abs(Yf - Yd)) <= 1e-12 * np.max(np.abs(Yd))


def test_circulant_embedding_masked_gap():
    prob = synth.make_problem(5, 3, 3, 10, seed=3, gap_column=2, edge_layout="split",
                              rhs="planewave", nrhs=2)
    Yd = oracle.matvec_dense(oracle.assemble(prob), prob.V)
    Yf = fft_embedded_matvec(prob, prob.V, 9, 6)
    assert np.max(np.abs(Yf - Yd)) <= 1e-12 * np.max(np.abs(Yd))


def test_matvec_blocks_and_rows_equal_dense():
    for prob in small_problems():
        Z = oracle.assemble(prob)
        Yd = oracle.matvec_dense(Z, prob.V)
        Yb = oracle.matvec_blocks(prob, prob.V)
        assert np.max(np.abs(Yb - Yd)) <= 1e-13 * np.max(np.abs(Yd))
        rows = np.array([0, prob.n - 1, prob.n // 2])
        Yr = oracle.matvec_rows(prob, prob.V, rows)
        assert np.max(np.abs(Yr - Yd[:, rows])) <= 1e-13 * np.max(np.abs(Yd))


def test_toeplitz_index_rule_brute_force():
    # Eq. submatrixAA: block (row part (m,n), column part (m',n')) of A is the
    # generating block of offset (m-m', n-n'); x fastest inside y.
    prob = synth.make_problem(3, 2, 2, 3, seed=6)
    Z = oracle.assemble(prob)
    nx, ny, b = prob.nx, prob.ny, prob.b
    for n in range(ny):
        for m in range(nx):
            for n2 in range(ny):
                for m2 in range(nx):
                    for i in range(b):
                        for j in range(b):
                            k = (n * nx + m) * b + i
                            l = (n2 * nx + m2) * b + j
                            assert Z[k, l] == prob.T[n - n2 + ny - 1, m - m2 + nx - 1, i, j]


# ---------------------------------------------------------------- solves

def test_lu_matches_lapack_and_residual():
    for prob in [synth.make_problem(4, 4, 8, 16, seed=0),
                 synth.make_problem(6, 5, 12, 40, seed=4, rhs="planewave", nrhs=4)]:
        Z = oracle.assemble(prob)
        lu = oracle.LU(Z)
        X = lu.solve(prob.V)
        Xl = np.linalg.solve(Z, prob.V.T).T
        assert np.max(np.abs(X - Xl)) <= 1e-11 * np.max(np.abs(Xl))
        assert oracle.relres(Z, X, prob.V).max() <= 1e-13


def test_lu_diagonal_closed_form():
    # T = c * delta_{p,q,0} * I, no edges: Z = c I, so x = v / c.
    prob = synth.make_problem(3, 3, 4, 0, seed=1, rhs="planewave", nrhs=2)
    c = 2.0 - 0.75j
    prob.T[:] = 0
    prob.T[2, 2] = c * np.eye(4)
    X = oracle.LU(oracle.assemble(prob)).solve(prob.V)
    assert np.allclose(X, prob.V / c, rtol=1e-15, atol=0)


def test_cond_estimate_against_exact():
    prob = synth.make_problem(4, 4, 8, 16, seed=0)
    Z = oracle.assemble(prob)
    est = oracle.LU(Z).cond1_estimate()
    exact = np.linalg.cond(Z, 1)
    assert exact / 3 <= est <= exact * (1 + 1e-10)


def test_schur_complement_equals_monolithic():
    # Sec. II-D: I1 = U - F I2, I2 = -(C - B F)^-1 B U with A [U F] = [V1 B^T].
    prob = synth.make_problem(3, 3, 6, 12, seed=9, rhs="ports")
    Z = oracle.assemble(prob)
    nt = prob.n_toep
    A = Z[:nt, :nt]
    X = oracle.schur_solve(A, prob.B, prob.C, prob.V)
    Xm = oracle.LU(Z).solve(prob.V)
    assert np.max(np.abs(X - Xm)) <= 1e-11 * np.max(np.abs(Xm))
    # V = [V1; 0] port excitation: i_n = i_1 + (n-1) e5 with e5 = b (Sec. II-D)
    ports = np.nonzero(prob.V)[1]
    assert np.array_equal(ports, np.arange(prob.nx * prob.ny) * prob.b)


def test_masked_elements_solution_exactly_zero():
    prob = synth.make_problem(5, 3, 3, 10, seed=3, gap_column=2, edge_layout="split",
                              rhs="planewave", nrhs=2)
    mask = oracle.unknown_mask(prob)
    V = prob.V * mask[None, :]
    X = oracle.LU(oracle.assemble(prob)).solve(V)
    assert np.all(X[:, mask == 0] == 0)


def test_oracle_gmres_converges_to_lu_solution():
    prob = synth.make_problem(4, 4, 8, 16, seed=0)
    Z = oracle.assemble(prob)
    xl = oracle.LU(Z).solve(prob.V)[0]
    x, its, rel = oracle.gmres(prob, prob.V[0], restart=30, tol=1e-12, max_iter=500)
    assert rel <= 1e-12 and its < 500
    assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= 1e-10


# ---------------------------------------------------------------- perimeter side layout
def _side_edge(nx, ny, k, sg, c, s):
    """Edge index of (side, cell, sub-position) in the counter-clockwise layout:
    bottom (left to right), right (upwards), top and left stored in reverse."""
    lens = (nx, ny, nx, ny)
    base = (0, k * nx, k * (nx + ny), k * (2 * nx + ny))[sg]
    if sg < 2:
        return base + k * c + s
    return base + k * (lens[sg] - 1 - c) + (k - 1 - s)


@pytest.mark.parametrize("nx,ny,k", [(4, 4, 1), (6, 5, 2), (5, 7, 3), (3, 2, 4)])
def test_perimeter_layout_positions_and_side_toeplitz(nx, ny, k):
    """The perimeter points of the 'one' layout with E = 2k(nx+ny) sit at
    (c + (s + 1/2)/k) a along each side, and each side's block of B depends on
    the element only through c - m (bottom/top) or c - n (right/left): the
    one-level block-Toeplitz side blocks of Sec. II-C (Eqs. submatrixB12/B34)."""
    a = synth.PERIOD
    prob = synth.make_problem(nx, ny, 5, 2 * k * (nx + ny), seed=4)
    assert prob.edge_per_cell == k
    for sg in range(4):
        L = nx if sg % 2 == 0 else ny
        for c in range(L):
            for s in range(k):
                along = (c + (s + 0.5) / k) * a
                expect = [(along, 0.0), (nx * a, along), (along, ny * a), (0.0, along)][sg]
                e = _side_edge(nx, ny, k, sg, c, s)
                assert np.allclose(prob.edge_pts[e], expect, rtol=0, atol=1e-12)
    B = prob.B.reshape(prob.n_edge, ny, nx, prob.b)  # [e][n][m][i]
    scale = np.abs(B).max()
    for sg in range(4):
        L = nx if sg % 2 == 0 else ny
        for s in range(k):
            for c in range(L):
                for c2 in range(L):
                    d = c2 - c  # shifting the cell and the element by the same d
                    e1, e2 = _side_edge(nx, ny, k, sg, c, s), _side_edge(nx, ny, k, sg, c2, s)
                    if sg % 2 == 0:
                        lo, hi = max(0, -d), min(nx, nx - d)
                        if lo < hi:
                            assert np.max(np.abs(B[e1, :, lo:hi] - B[e2, :, lo + d:hi + d])) <= 1e-12 * scale
                    else:
                        lo, hi = max(0, -d), min(ny, ny - d)
                        if lo < hi:
                            assert np.max(np.abs(B[e1, lo:hi] - B[e2, lo + d:hi + d])) <= 1e-12 * scale


def test_edge_per_cell_only_for_the_full_perimeter_layout():
    assert synth.make_problem(4, 4, 3, 16).edge_per_cell == 1
    assert synth.make_problem(4, 4, 3, 15).edge_per_cell == 0
    assert synth.make_problem(4, 4, 3, 0).edge_per_cell == 0
    p = synth.make_problem(5, 3, 3, 16, gap_column=2, edge_layout="split")
    assert p.edge_per_cell == 0


# ---- port matrices (Sec. IV-B)

def test_port_scattering_one_port_closed_form():
    """One port: S = (1/y - z0) / (1/y + z0) (F cancels for a 1 x 1 matrix)."""
    for y, z0 in ((0.013 - 0.004j, 50.0), (2.0 + 1.0j, 0.7)):
        S = oracle.scattering(np.array([[y]]), np.array([z0]))
        assert S.shape == (1, 1)
        assert abs(S[0, 0] - (1 / y - z0) / (1 / y + z0)) <= 1e-14


def test_port_scattering_terminations():
    """Matched ports (Z_port = diag(z0)) reflect nothing; near-open ports
    (Y -> 0) give S -> I; near-short ports (Y -> inf) give S -> -I."""
    z0 = np.array([50.0, 75.0, 20.0])
    assert np.max(np.abs(oracle.scattering(np.diag(1 / z0), z0))) <= 1e-14
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    assert np.max(np.abs(oracle.scattering(1e-9 * Y, z0) - np.eye(3))) <= 1e-6
    assert np.max(np.abs(oracle.scattering(1e9 * Y, z0) + np.eye(3))) <= 1e-6


@pytest.mark.parametrize("uniform", [True, False])
def test_port_scattering_lossless_is_unitary(uniform):
    """A lossless reciprocal network (Z_port = j X, X real symmetric) has a
    unitary, and for equal reference impedances symmetric, power-wave S; with
    unequal real z0 unitarity needs the F scaling."""
    rng = np.random.default_rng(4)
    p = 6
    A = rng.standard_normal((p, p))
    X = 30.0 * (A + A.T)
    z0 = np.full(p, 50.0) if uniform else rng.uniform(20.0, 100.0, p)
    S = oracle.scattering(np.linalg.inv(1j * X), z0)
    assert np.max(np.abs(S.conj().T @ S - np.eye(p))) <= 1e-10
    if uniform:
        assert np.max(np.abs(S - S.T)) <= 1e-10


def test_port_admittance_is_the_port_block_of_the_inverse():
    """Delta-port solutions of the dense system: I^ = (Z^-1) restricted to
    the port rows and columns, so Y = L (Z^-1)[ports, ports] L, symmetric
    because the MoM matrix is (Galerkin, Z^T = Z)."""
    prob = synth.make_problem(4, 3, 5, 8, seed=2)
    Z = oracle.assemble(prob)
    ports = np.array([0, 7, 23, 40, prob.n - 1])
    lens = np.array([0.5, 0.25, 1.0, 0.75, 2.0])
    V = np.zeros((len(ports), prob.n), complex)
    V[np.arange(len(ports)), ports] = 1.0
    I = np.linalg.solve(Z, V.T).T  # row k: solution for port k
    Y = oracle.port_admittance(I, ports, lens)
    Zi = np.linalg.inv(Z)
    L = np.diag(1 / lens)
    assert np.max(np.abs(Y - L @ Zi[np.ix_(ports, ports)] @ L)) <= 1e-12 * np.max(np.abs(Y))
    assert np.max(np.abs(Y - Y.T)) <= 1e-12 * np.max(np.abs(Y))


# ---- far field (Eqs. farfieldBasis / tensorProd)

def test_far_field_single_element_closed_form():
    """One element at the origin: no phase, F = -j k eta sum_i I_i Fh[m][t][i]."""
    prob = synth.make_problem(1, 1, 3, 0, seed=6)
    rng = np.random.default_rng(0)
    I = rng.standard_normal((2, 3)) + 1j * rng.standard_normal((2, 3))
    uv = rng.uniform(-1, 1, (5, 2))
    Fh = rng.standard_normal((5, 2, 3)) + 1j * rng.standard_normal((5, 2, 3))
    F = oracle.far_field(prob, I, uv, Fh, k=2.0, eta=3.0)
    ref = -1j * 2.0 * 3.0 * np.einsum("mti,ri->rmt", Fh, I)
    assert np.max(np.abs(F - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_far_field_shift_theorem():
    """Moving the currents of element (0, 0) to element (1, 1) multiplies the
    far field by exp(j k a (u + v)) (the offset d = (a, a, 0))."""
    prob = synth.make_problem(3, 2, 4, 0, seed=1)
    rng = np.random.default_rng(3)
    c = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    I0 = np.zeros((1, prob.n_toep), complex)
    I1 = np.zeros((1, prob.n_toep), complex)
    I0[0, 0:4] = c
    p = 1 * prob.nx + 1
    I1[0, 4 * p:4 * p + 4] = c
    uv = rng.uniform(-1, 1, (7, 2))
    Fh = synth.far_field_basis(prob, uv)
    k = synth.K0
    F0 = oracle.far_field(prob, I0, uv, Fh, k, 1.0)
    F1 = oracle.far_field(prob, I1, uv, Fh, k, 1.0)
    ph = np.exp(1j * k * synth.PERIOD * (uv[:, 0] + uv[:, 1]))
    assert np.max(np.abs(F1 - F0 * ph[None, :, None])) <= 1e-13 * np.max(np.abs(F0))


def test_far_field_on_the_grid_is_an_inverse_fft():
    """On the array-factor grid of an lx x ly embedding the sum over parts is
    lx ly times numpy's inverse 2-D FFT of the zero-padded element currents
    (per basis function), contracted with Fh."""
    prob = synth.make_problem(5, 3, 2, 0, seed=4, gap_column=2)
    lx, ly = 9, 6
    rng = np.random.default_rng(5)
    I = rng.standard_normal((2, prob.n_toep)) + 1j * rng.standard_normal((2, prob.n_toep))
    uv = synth.grid_directions(lx, ly)
    Fh = synth.far_field_basis(prob, uv)
    F = oracle.far_field(prob, I, uv, Fh, synth.K0, 120 * np.pi)
    grid = I.reshape(2, prob.ny, prob.nx, prob.b) * prob.active[None, :, :, None]
    pad = np.zeros((2, ly, lx, prob.b), complex)
    pad[:, :prob.ny, :prob.nx] = grid
    Xs = np.fft.ifft2(pad, axes=(1, 2)) * (lx * ly)          # [r][ky][kx][i], e^{+j...}
    ref = -1j * synth.K0 * 120 * np.pi * np.einsum("fti,rfi->rft", Fh, Xs.reshape(2, ly * lx, prob.b))
    assert np.max(np.abs(F - ref)) <= 1e-11 * np.max(np.abs(ref))
