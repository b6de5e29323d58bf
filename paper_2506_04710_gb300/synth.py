"""Seeded synthetic inputs for the two-level block-Toeplitz array system.

This module only *generates inputs*: basis points, the generating blocks
T[p,q] of the element-to-element matrix A, the edge-coupling blocks B and C,
the activity mask and right-hand sides.  It holds none of the solver's
arithmetic (no embedding, FFT, product or Krylov step).  Both the CUDA path
and the CPU oracle consume the arrays it returns.

Physics stand-in (the paper's RWG meshes and DEMCEM integrals are not
available): every matrix entry is the free-space Green's function of Sec. II,
G(R) = exp(-jkR)/(4 pi R), evaluated between point-like basis functions, with
R regularised to R' = max(R, 0.05 lambda) in both the phase and the 1/R, and
with (1 + 0.5j) added on the global diagonal.  lambda = 1, k = 2 pi, the
array period is a = 0.5 lambda and the element basis points are uniform in
the a x a cell.

Random numbers: a counter-based SplitMix64 stream (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014).  Draw k of
stream s under seed sigma is mix64(s0 + (k+1) * GAMMA) with
s0 = sigma + s * STREAM_KEY (mod 2**64); a double in [0,1) takes the top 53
bits.  Stream 0 holds the basis points (u_0, v_0, u_1, v_1, ...), stream 1
the plane-wave angles (theta_0, phi_0, ...), stream 2 manufactured solutions,
stream 3 serving-request parameters.

Unknown ordering (Sec. II-C, part indexing of component 5 with x fastest,
and the block form [[A, B^T], [B, C]]): Toeplitz unknown (m, n, i) of element
column m, row n and local basis i has index (n*Nx + m)*b + i; the E edge
unknowns follow at N_T .. N_T+E-1.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LAMBDA = 1.0
K0 = 2.0 * math.pi / LAMBDA
PERIOD = 0.5 * LAMBDA
R_MIN = 0.05 * LAMBDA
DIAG = 1.0 + 0.5j

GAMMA = np.uint64(0x9E3779B97F4A7C15)
STREAM_KEY = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_POINTS = 0
STREAM_ANGLES = 1
STREAM_MANUFACTURED = 2
STREAM_REQUESTS = 3


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+n-1 of stream `stream` under `seed`, in [0, 1)."""
    with np.errstate(over="ignore"):
        s0 = np.uint64(seed % (1 << 64)) + np.uint64(stream) * STREAM_KEY
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = _mix64(s0 + k * GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def green_reg(R: np.ndarray) -> np.ndarray:
    """Regularised Green's function exp(-jkR')/(4 pi R'), R' = max(R, R_MIN)."""
    Rp = np.maximum(R, R_MIN)
    return np.exp(-1j * K0 * Rp) / (4.0 * math.pi * Rp)


@dataclasses.dataclass
class Problem:
    """One synthetic array system.  Arrays are complex128 / float64 / uint8.

    T: [2Ny-1][2Nx-1][b][b]; T[q+Ny-1][p+Nx-1] is the block for element offset
       (p, q) = (m-m', n-n').
    B: [E][N_T] coupling of edge unknown e with Toeplitz unknown t.
    C: [E][E].
    active: [Ny][Nx] (1 = element present).
    V: [nrhs][N] right-hand sides (rows of the array are RHS columns).
    pts: [b][2] element basis points; edge_pts: [E][2].
    """
    nx: int
    ny: int
    b: int
    n_edge: int
    seed: int
    T: np.ndarray
    B: np.ndarray
    C: np.ndarray
    active: np.ndarray
    V: np.ndarray
    pts: np.ndarray
    edge_pts: np.ndarray
    name: str = ""
    edge_layout: str = "one"

    @property
    def n_toep(self) -> int:
        return self.nx * self.ny * self.b

    @property
    def n(self) -> int:
        return self.n_toep + self.n_edge

    @property
    def nrhs(self) -> int:
        return self.V.shape[0]

    @property
    def edge_per_cell(self) -> int:
        """k when the edge unknowns are k per cell side on the whole perimeter
        (E = 2k(Nx + Ny), equal spacing a/k from half a spacing after (0, 0)),
        else 0."""
        per = 2 * (self.nx + self.ny)
        if self.n_edge == 0 or self.n_edge % per or self.edge_layout != "one":
            return 0
        return self.n_edge // per


def basis_points(seed: int, b: int) -> np.ndarray:
    u = uniform(seed, STREAM_POINTS, 2 * b).reshape(b, 2)
    return PERIOD * u


def perimeter_points(x0: float, y0: float, w: float, h: float, count: int) -> np.ndarray:
    """`count` points at equal arc length on the rectangle boundary, counter-clockwise
    from (x0, y0), the first one half a spacing from the corner."""
    if count == 0:
        return np.zeros((0, 2))
    per = 2.0 * (w + h)
    s = (np.arange(count, dtype=np.float64) + 0.5) * (per / count)
    out = np.empty((count, 2))
    for k, t in enumerate(s):
        if t < w:
            out[k] = (x0 + t, y0)
        elif t < w + h:
            out[k] = (x0 + w, y0 + (t - w))
        elif t < 2 * w + h:
            out[k] = (x0 + w - (t - w - h), y0 + h)
        else:
            out[k] = (x0, y0 + h - (t - 2 * w - h))
    return out


def toeplitz_blocks(pts: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """T[q+ny-1][p+nx-1][i][j] = G_reg(|r_i - r_j + (p a, q a)|) (+DIAG on the
    global diagonal).  dx is formed as (x_i - x_j) + p*a so that the block of
    (-p, -q) is bitwise the transpose of the block of (p, q)."""
    b = pts.shape[0]
    dxs = pts[:, None, 0] - pts[None, :, 0]
    dys = pts[:, None, 1] - pts[None, :, 1]
    T = np.empty((2 * ny - 1, 2 * nx - 1, b, b), dtype=np.complex128)
    for q in range(-(ny - 1), ny):
        dy = dys + q * PERIOD
        for p in range(-(nx - 1), nx):
            dx = dxs + p * PERIOD
            T[q + ny - 1, p + nx - 1] = green_reg(np.sqrt(dx * dx + dy * dy))
    idx = np.arange(b)
    T[ny - 1, nx - 1, idx, idx] += DIAG
    return T


def toeplitz_positions(pts: np.ndarray, nx: int, ny: int) -> np.ndarray:
    """[N_T][2] positions of the Toeplitz unknowns in index order (n*Nx+m)*b+i."""
    b = pts.shape[0]
    m = np.arange(nx)
    n = np.arange(ny)
    X = np.broadcast_to(m[None, :, None] * PERIOD + pts[None, None, :, 0], (ny, nx, b))
    Y = np.broadcast_to(n[:, None, None] * PERIOD + pts[None, None, :, 1], (ny, nx, b))
    return np.stack([X.reshape(-1), Y.reshape(-1)], axis=1)


def edge_blocks(pts: np.ndarray, nx: int, ny: int, edge_pts: np.ndarray,
                chunk: int = 64) -> tuple[np.ndarray, np.ndarray]:
    """B[e][(n*Nx+m)*b+i] = G_reg(|p_e - (r_i + (m a, n a))|), C[e][e'] = G_reg(|p_e-p_e'|)+DIAG*delta."""
    pos = toeplitz_positions(pts, nx, ny)
    E = edge_pts.shape[0]
    B = np.empty((E, pos.shape[0]), dtype=np.complex128)
    for e0 in range(0, E, chunk):
        e1 = min(E, e0 + chunk)
        dx = edge_pts[e0:e1, None, 0] - pos[None, :, 0]
        dy = edge_pts[e0:e1, None, 1] - pos[None, :, 1]
        B[e0:e1] = green_reg(np.sqrt(dx * dx + dy * dy))
    dx = edge_pts[:, None, 0] - edge_pts[None, :, 0]
    dy = edge_pts[:, None, 1] - edge_pts[None, :, 1]
    C = green_reg(np.sqrt(dx * dx + dy * dy))
    C[np.arange(E), np.arange(E)] += DIAG
    return B, C


def unknown_positions(prob: Problem) -> np.ndarray:
    return np.concatenate([toeplitz_positions(prob.pts, prob.nx, prob.ny), prob.edge_pts])


def plane_waves(positions: np.ndarray, seed: int, nrhs: int) -> np.ndarray:
    """v_k = exp(+jk(sin t cos f x_k + sin t sin f y_k)), t ~ U[0, 60 deg], f ~ U[0, 360 deg)."""
    u = uniform(seed, STREAM_ANGLES, 2 * nrhs).reshape(nrhs, 2)
    theta = u[:, 0] * (math.pi / 3.0)
    phi = u[:, 1] * (2.0 * math.pi)
    kx = K0 * np.sin(theta) * np.cos(phi)
    ky = K0 * np.sin(theta) * np.sin(phi)
    return np.exp(1j * (kx[:, None] * positions[None, :, 0] + ky[:, None] * positions[None, :, 1]))


def make_problem(nx: int, ny: int, b: int, n_edge: int, seed: int = 0, rhs: str = "ones",
                 nrhs: int = 1, gap_column: int | None = None, edge_layout: str = "one",
                 name: str = "") -> Problem:
    """Build a seeded problem.

    rhs: "ones" (unit amplitude, uniform phase on all N unknowns), "ports"
    (one unit delta per active element at its local basis 0, element order
    (n, m); edge rows zero) or "planewave" (nrhs seeded scan angles).
    edge_layout: "one" = n_edge points on the whole array perimeter; "split" =
    half on each of the two sub-array perimeters left and right of gap_column.
    """
    pts = basis_points(seed, b)
    active = np.ones((ny, nx), dtype=np.uint8)
    if gap_column is not None:
        active[:, gap_column] = 0
    if edge_layout == "one":
        edge_pts = perimeter_points(0.0, 0.0, nx * PERIOD, ny * PERIOD, n_edge)
    elif edge_layout == "split":
        assert gap_column is not None and n_edge % 2 == 0
        left = perimeter_points(0.0, 0.0, gap_column * PERIOD, ny * PERIOD, n_edge // 2)
        right = perimeter_points((gap_column + 1) * PERIOD, 0.0,
                                 (nx - gap_column - 1) * PERIOD, ny * PERIOD, n_edge // 2)
        edge_pts = np.concatenate([left, right])
    else:
        raise ValueError(edge_layout)
    T = toeplitz_blocks(pts, nx, ny)
    B, C = edge_blocks(pts, nx, ny, edge_pts)
    nt = nx * ny * b
    N = nt + n_edge
    if rhs == "ones":
        V = np.ones((nrhs, N), dtype=np.complex128)
    elif rhs == "ports":
        els = [(n * nx + m) for n in range(ny) for m in range(nx) if active[n, m]]
        V = np.zeros((len(els), N), dtype=np.complex128)
        for k, el in enumerate(els):
            V[k, el * b] = 1.0
    elif rhs == "planewave":
        pos = np.concatenate([toeplitz_positions(pts, nx, ny), edge_pts])
        V = plane_waves(pos, seed, nrhs)
    else:
        raise ValueError(rhs)
    return Problem(nx, ny, b, n_edge, seed, T, B, C, active, V, pts, edge_pts, name, edge_layout)


def manufactured_solution(prob: Problem, nrhs: int, seed: int | None = None) -> np.ndarray:
    """Seeded x* [nrhs][N] with entries uniform in the unit square of C, zero on
    inactive elements (their rows are identity rows with zero RHS)."""
    s = prob.seed if seed is None else seed
    u = uniform(s, STREAM_MANUFACTURED, 2 * nrhs * prob.n).reshape(nrhs, prob.n, 2)
    x = (u[..., 0] - 0.5) + 1j * (u[..., 1] - 0.5)
    mask = np.concatenate([np.repeat(prob.active.reshape(-1), prob.b), np.ones(prob.n_edge, np.uint8)])
    return x * mask[None, :]


# The workloads: grid, basis count, edge unknowns, RHS recipe.
CONFIGS = {
    "c1_4x4_b8": dict(nx=4, ny=4, b=8, n_edge=16, rhs="ones", nrhs=1, tol=1e-10),
    "c2_32x32_b64": dict(nx=32, ny=32, b=64, n_edge=512, rhs="ones", nrhs=1, tol=1e-8),
    "c3_19x9gap_b48": dict(nx=19, ny=9, b=48, n_edge=324, rhs="ports", nrhs=162, gap_column=9,
                           edge_layout="split", tol=1e-8),
    "c4_64x64_b96": dict(nx=64, ny=64, b=96, n_edge=1024, rhs="planewave", nrhs=32, tol=1e-8),
}


def config_problem(key: str, seed: int = 0) -> tuple[Problem, float]:
    cfg = dict(CONFIGS[key])
    tol = cfg.pop("tol")
    return make_problem(seed=seed, name=key, **cfg), tol


def serving_requests(n: int = 2000, rate: float = 50.0, seed: int = 0,
                     sizes=(8, 48), bases=(32, 48, 64, 96), max_rhs: int = 64, designs: int = 4):
    """Poisson stream: (arrival_s, nx, b, nrhs, req_seed).  Square arrays,
    E = 16*Nx edge unknowns, plane-wave RHS.  The request seed (which fixes
    the element geometry, hence the generating blocks) is one of `designs`
    values, so requests for the same (Nx, b, seed) design share a plan."""
    u = uniform(seed, STREAM_REQUESTS, 5 * n).reshape(n, 5)
    gaps = -np.log1p(-u[:, 0]) / rate
    t = np.cumsum(gaps)
    nx = sizes[0] + np.minimum((u[:, 1] * (sizes[1] - sizes[0] + 1)).astype(int), sizes[1] - sizes[0])
    b = np.array(bases)[np.minimum((u[:, 2] * len(bases)).astype(int), len(bases) - 1)]
    nrhs = 1 + np.minimum((u[:, 3] * max_rhs).astype(int), max_rhs - 1)
    rseed = 1000 + np.minimum((u[:, 4] * designs).astype(np.int64), designs - 1)
    return [(float(t[k]), int(nx[k]), int(b[k]), int(nrhs[k]), int(rseed[k])) for k in range(n)]


# ---------------------------------------------------------------- device-side generation
# The same recipe evaluated with torch on a CUDA device, for request streams
# whose host generation would take longer than the arrival interval.  Draws
# come from the same SplitMix64 streams (on the host, O(b) numbers); the
# Green's function values agree with the NumPy ones to rounding.

def _green_torch(R):
    import torch
    Rp = torch.clamp(R, min=R_MIN)
    return torch.exp(-1j * K0 * Rp.to(torch.complex128)) / (4.0 * math.pi * Rp)


def make_problem_device(nx: int, ny: int, b: int, n_edge: int, seed: int, nrhs: int, device="cuda",
                        chunk_elems: int = 1 << 26) -> dict:
    """Square-cell array with edge points on its perimeter and plane-wave RHS,
    as torch tensors on `device`: T [2ny-1][2nx-1][b][b], B [E][N_T], C [E][E],
    V [nrhs][N] (complex128)."""
    import torch
    pts_np = basis_points(seed, b)
    pts = torch.from_numpy(pts_np).to(device)
    dxs = pts[:, None, 0] - pts[None, :, 0]
    dys = pts[:, None, 1] - pts[None, :, 1]
    p = torch.arange(-(nx - 1), nx, device=device, dtype=torch.float64) * PERIOD
    q = torch.arange(-(ny - 1), ny, device=device, dtype=torch.float64) * PERIOD
    dx = dxs[None, None] + p[None, :, None, None]
    dy = dys[None, None] + q[:, None, None, None]
    T = _green_torch(torch.sqrt(dx * dx + dy * dy))
    idx = torch.arange(b, device=device)
    T[ny - 1, nx - 1, idx, idx] += DIAG
    edge_np = perimeter_points(0.0, 0.0, nx * PERIOD, ny * PERIOD, n_edge)
    pos_np = toeplitz_positions(pts_np, nx, ny)
    pos = torch.from_numpy(np.ascontiguousarray(pos_np)).to(device)
    edge = torch.from_numpy(edge_np).to(device)
    nt = pos.shape[0]
    B = torch.empty((n_edge, nt), dtype=torch.complex128, device=device)
    rows = max(1, chunk_elems // max(1, nt))
    for e0 in range(0, n_edge, rows):
        e1 = min(n_edge, e0 + rows)
        ddx = edge[e0:e1, None, 0] - pos[None, :, 0]
        ddy = edge[e0:e1, None, 1] - pos[None, :, 1]
        B[e0:e1] = _green_torch(torch.sqrt(ddx * ddx + ddy * ddy))
    ddx = edge[:, None, 0] - edge[None, :, 0]
    ddy = edge[:, None, 1] - edge[None, :, 1]
    C = _green_torch(torch.sqrt(ddx * ddx + ddy * ddy))
    C[torch.arange(n_edge, device=device), torch.arange(n_edge, device=device)] += DIAG
    u = uniform(seed, STREAM_ANGLES, 2 * nrhs).reshape(nrhs, 2)
    theta = u[:, 0] * (math.pi / 3.0)
    phi = u[:, 1] * (2.0 * math.pi)
    kx = torch.from_numpy(K0 * np.sin(theta) * np.cos(phi)).to(device)
    ky = torch.from_numpy(K0 * np.sin(theta) * np.sin(phi)).to(device)
    allpos = torch.cat([pos, edge])
    ph = kx[:, None] * allpos[None, :, 0] + ky[:, None] * allpos[None, :, 1]
    V = torch.exp(1j * ph.to(torch.complex128))
    return dict(nx=nx, ny=ny, b=b, n_edge=n_edge, T=T.contiguous(), B=B, C=C.contiguous(), V=V.contiguous())


def grid_directions(lx: int, ly: int, period: float = PERIOD) -> np.ndarray:
    """Observation directions (u, v) = (sin th cos ph, sin th sin ph) of the
    array-factor grid of an lx x ly embedding, in the spectrum's order
    f = ky lx + kx: u = kx' lambda / (lx a), v = ky' lambda / (ly a), with
    kx' = kx for kx <= lx / 2 and kx - lx above (so k a u m = 2 pi kx m / lx
    for every integer m).  Points with u^2 + v^2 > 1 lie outside the visible
    region; they are kept (evanescent directions) so that the grid is whole."""
    kx = np.arange(lx)
    ky = np.arange(ly)
    kxs = np.where(kx <= lx // 2, kx, kx - lx)
    kys = np.where(ky <= ly // 2, ky, ky - ly)
    u = kxs * LAMBDA / (lx * period)
    v = kys * LAMBDA / (ly * period)
    U, V = np.meshgrid(u, v)
    return np.stack([U.reshape(-1), V.reshape(-1)], axis=1)


def far_field_basis(prob: "Problem", uv: np.ndarray, npol: int = 2) -> np.ndarray:
    """Synthetic stand-in for the per-basis far-field integrals of one element
    (the tensor F^[m][pol][i] of the paper's far-field step; the mesh
    integrals are not available): a point-like basis at r_i radiates
    exp(j k r^.r_i) times a smooth polarisation factor, 1 (co) and u v (cross).
    Returns complex128 [M][npol][b]."""
    uv = np.asarray(uv, dtype=np.float64)
    ph = np.exp(1j * K0 * (uv[:, 0:1] * prob.pts[None, :, 0] + uv[:, 1:2] * prob.pts[None, :, 1]))
    pol = [np.ones(len(uv)), uv[:, 0] * uv[:, 1]] + [uv[:, 0] ** q for q in range(2, npol)]
    return np.stack([pol[t][:, None] * ph for t in range(npol)], axis=1)
