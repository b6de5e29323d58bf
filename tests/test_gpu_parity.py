"""Parity of the CUDA path (through the C-ABI) with the CPU FP64 oracle on
small seeded systems: several tiles, ragged tails, odd and explicit embedding
sizes, masked elements, no edges, a single element, b = 1.

Tolerances:
  FP64 products: max-norm error <= 1e-12 relative to max |y| (rounding of an
    O(F log F) FFT chain on O(1) data; the paper's entries are complex128).
  MIXED products: per-RHS 2-norm error <= 2e-6 relative (FP32, u = 6e-8,
    times the FFT depth and the block-product length, with margin).
  Solves: true relative residual (recomputed by the oracle) <= the requested
    tol; solution error against the oracle's LU solve <= 1e-7 when solved to
    1e-11 (forward error <= cond * residual, cond <= 60 on these systems).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


CASES = {
    "4x4_b8_e16": dict(nx=4, ny=4, b=8, n_edge=16),
    "3x5_b4_e12_pw3": dict(nx=3, ny=5, b=4, n_edge=12, rhs="planewave", nrhs=3, seed=7),
    "5x3_b3_gap": dict(nx=5, ny=3, b=3, n_edge=10, gap_column=2, edge_layout="split", rhs="ports", seed=3),
    "1x1_b6_e5": dict(nx=1, ny=1, b=6, n_edge=5, seed=11),
    "2x3_b1_e0": dict(nx=2, ny=3, b=1, n_edge=0, rhs="planewave", nrhs=2, seed=5),
    "7x6_b12_e20": dict(nx=7, ny=6, b=12, n_edge=20, rhs="planewave", nrhs=5, seed=9),
    "9x4_b40_e24": dict(nx=9, ny=4, b=40, n_edge=24, rhs="planewave", nrhs=6, seed=13),
    "6x6_b33_e0_gap": dict(nx=6, ny=6, b=33, n_edge=0, gap_column=3, rhs="planewave", nrhs=2, seed=17),
    # more edge rows than the FP32 edge kernel stages at once (1024)
    "6x5_b4_e1100": dict(nx=6, ny=5, b=4, n_edge=1100, rhs="planewave", nrhs=3, seed=19),
}


def make(key):
    kw = dict(CASES[key])
    return synth.make_problem(**kw)


def embedded_spectrum(prob, lx, ly):
    emb = np.zeros((ly, lx, prob.b, prob.b), complex)
    for q in range(-(prob.ny - 1), prob.ny):
        for p in range(-(prob.nx - 1), prob.nx):
            emb[q % ly, p % lx] = prob.T[q + prob.ny - 1, p + prob.nx - 1]
    return np.fft.fft2(emb, axes=(0, 1))


@pytest.mark.parametrize("key", list(CASES))
def test_plan_spectrum_matches_numpy_fft(key):
    prob = make(key)
    plan = ztoep.Plan.from_problem(prob)
    lx, ly = plan.info.lx, plan.info.ly
    assert lx == synth_smooth(2 * prob.nx - 1) and ly == synth_smooth(2 * prob.ny - 1)
    That = torch.empty((lx * ly, prob.b, prob.b), dtype=torch.complex128, device="cuda")
    assert ztoep.ztoep_plan_spectrum(plan.handle, That) == 0
    ref = embedded_spectrum(prob, lx, ly).reshape(lx * ly, prob.b, prob.b)
    got = host(That)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    plan.close()


def synth_smooth(n):
    L = max(1, n)
    while True:
        k = L
        for q in (2, 3, 5):
            while k % q == 0:
                k //= q
        if k == 1:
            return L
        L += 1


@pytest.mark.parametrize("key", ["4x4_b8_e16", "5x3_b3_gap", "9x4_b40_e24", "2x3_b1_e0"])
@pytest.mark.parametrize("prec", [ztoep.ZTOEP_FP64, ztoep.ZTOEP_MIXED])
def test_forward_spectrum_matches_numpy_fft(key, prec):
    prob = make(key)
    plan = ztoep.Plan.from_problem(prob)
    lx, ly = plan.info.lx, plan.info.ly
    X = dev(prob.V)
    nr = prob.nrhs
    Xh = torch.empty((lx * ly, nr, prob.b), dtype=torch.complex128, device="cuda")
    assert ztoep.ztoep_forward_spectrum(plan.handle, prec, nr, X, Xh) == 0
    got = host(Xh)
    mask = np.repeat(prob.active.reshape(-1), prob.b)
    for r in range(nr):
        xt = (prob.V[r, :prob.n_toep] * mask).reshape(prob.ny, prob.nx, prob.b)
        pad = np.zeros((ly, lx, prob.b), complex)
        pad[:prob.ny, :prob.nx] = xt
        ref = np.fft.fft2(pad, axes=(0, 1)).reshape(lx * ly, prob.b)
        tol = 1e-12 if prec == ztoep.ZTOEP_FP64 else 2e-6
        assert np.max(np.abs(got[:, r] - ref)) <= tol * max(1e-300, np.max(np.abs(ref)))
    plan.close()


@pytest.mark.parametrize("key", list(CASES))
def test_matvec_fp64_vs_oracle(key):
    prob = make(key)
    ref = oracle.matvec_dense(oracle.assemble(prob), prob.V)
    plan = ztoep.Plan.from_problem(prob)
    got = host(plan.matvec(dev(prob.V), ztoep.ZTOEP_FP64))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    plan.close()


@pytest.mark.parametrize("key", list(CASES))
def test_matvec_mixed_vs_oracle(key):
    prob = make(key)
    ref = oracle.matvec_dense(oracle.assemble(prob), prob.V)
    plan = ztoep.Plan.from_problem(prob)
    got = host(plan.matvec(dev(prob.V), ztoep.ZTOEP_MIXED))
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-6
    plan.close()


@pytest.mark.parametrize("key,lx,ly", [("4x4_b8_e16", 8, 8), ("4x4_b8_e16", 9, 10),
                                       ("7x6_b12_e20", 15, 12), ("3x5_b4_e12_pw3", 5, 9)])
def test_matvec_explicit_embedding_sizes(key, lx, ly):
    prob = make(key)
    if not (synth_smooth(lx) == lx and synth_smooth(ly) == ly):
        pytest.skip("non-smooth size")
    ref = oracle.matvec_dense(oracle.assemble(prob), prob.V)
    plan = ztoep.Plan.from_problem(prob, lx=lx, ly=ly)
    assert plan.info.lx == lx and plan.info.ly == ly
    got = host(plan.matvec(dev(prob.V), ztoep.ZTOEP_FP64))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    plan.close()


def test_matvec_rejects_bad_arguments():
    prob = make("4x4_b8_e16")
    plan = ztoep.Plan.from_problem(prob)
    X = dev(prob.V)
    assert ztoep.ztoep_matvec(plan.handle, 7, 1, X, torch.empty_like(X)) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_matvec(plan.handle, 0, 0, X, torch.empty_like(X)) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_matvec(plan.handle, 0, 1, X, X) == ztoep.ZTOEP_ERR_ARG
    plan.close()


def opts(prec, tol, restart=30, max_iter=4000, inner_tol=1e-5):
    o = ztoep.ztoep_default_opts()
    o.prec, o.tol, o.restart, o.max_iter, o.inner_tol = prec, tol, restart, max_iter, inner_tol
    return o


@pytest.mark.parametrize("prec", [ztoep.ZTOEP_FP64, ztoep.ZTOEP_MIXED])
@pytest.mark.parametrize("key", ["4x4_b8_e16", "3x5_b4_e12_pw3", "5x3_b3_gap", "7x6_b12_e20", "9x4_b40_e24"])
def test_solve_vs_lu(key, prec):
    prob = make(key)
    Z = oracle.assemble(prob)
    mask = oracle.unknown_mask(prob)
    V = prob.V * mask[None, :]
    lu = oracle.LU(Z)
    Xref = lu.solve(V)
    plan = ztoep.Plan.from_problem(prob)
    # the config tolerance: the true residual must meet it
    tol = 1e-10 if prec == ztoep.ZTOEP_FP64 else 1e-8
    X, info, st = plan.solve(dev(V), opts=opts(prec, tol))
    assert st == 0
    res = oracle.relres(Z, host(X), V)
    assert res.max() <= tol
    for r, i in enumerate(info):
        assert i["status"] == 0 and i["rel_residual"] <= tol
        assert abs(i["rel_residual"] - res[r]) <= 1e-3 * tol + 1e-15
    # tightened: forward error against LU
    X2, info2, st2 = plan.solve(dev(V), opts=opts(prec, 1e-11))
    assert st2 == 0
    err = np.linalg.norm(host(X2) - Xref, axis=1) / np.linalg.norm(Xref, axis=1)
    assert err.max() <= 1e-7
    plan.close()


def test_masked_solution_exactly_zero():
    prob = make("5x3_b3_gap")
    mask = oracle.unknown_mask(prob)
    V = synth.plane_waves(synth.unknown_positions(prob), 3, 3) * mask[None, :]
    plan = ztoep.Plan.from_problem(prob)
    for prec in (ztoep.ZTOEP_FP64, ztoep.ZTOEP_MIXED):
        X, info, st = plan.solve(dev(V), opts=opts(prec, 1e-10))
        assert st == 0
        assert np.all(host(X)[:, mask == 0] == 0)
    plan.close()


def test_batch_equals_alone_bitwise():
    prob = make("7x6_b12_e20")
    plan = ztoep.Plan.from_problem(prob)
    V = dev(prob.V)
    Xb, _, _ = plan.solve(V, opts=opts(ztoep.ZTOEP_MIXED, 1e-8))
    for r in (0, 3):
        Xa, _, _ = plan.solve(V[r:r + 1].contiguous(), opts=opts(ztoep.ZTOEP_MIXED, 1e-8))
        assert torch.equal(Xa[0], Xb[r])
    plan.close()


def test_batch_equals_alone_across_reduction_modes():
    """20x20 b96 (N = 38,720: as many chunks as SMs, two-level Gram-Schmidt
    reductions over ten groups): one RHS alone and in a batch of 12 sum in
    the same order, so each solution is bitwise the same, in both precisions,
    and the batch meets the tolerance against the oracle."""
    prob = synth.make_problem(20, 20, 96, 320, seed=5, rhs="planewave", nrhs=12)
    plan = ztoep.Plan.from_problem(prob)
    V = dev(prob.V)
    for prec, tol in ((ztoep.ZTOEP_MIXED, 1e-8), (ztoep.ZTOEP_FP64, 1e-10)):
        Xb, _, st = plan.solve(V, opts=opts(prec, tol))
        assert st == 0
        for r in (0, 7, 11):
            Xa, _, _ = plan.solve(V[r:r + 1].contiguous(), opts=opts(prec, tol))
            assert torch.equal(Xa[0], Xb[r]), (prec, r)
    # the last batch is the FP64 one (tol 1e-10): every sampled residual
    # component is at most the residual's 2-norm
    rows = np.arange(0, prob.n, 97)
    res = oracle.matvec_rows(prob, Xb.cpu().numpy(), rows) - prob.V[:, rows]
    assert np.all(np.max(np.abs(res), axis=1) <= 2e-10 * np.linalg.norm(prob.V, axis=1))
    plan.close()


def test_solve_statuses():
    prob = make("7x6_b12_e20")
    plan = ztoep.Plan.from_problem(prob)
    V = prob.V.copy()
    V[2, 5] = np.nan
    X, info, st = plan.solve(dev(V), opts=opts(ztoep.ZTOEP_MIXED, 1e-8), check=False)
    assert st == ztoep.ZTOEP_ERR_NONFINITE
    assert info[2]["status"] == ztoep.ZTOEP_ERR_NONFINITE
    assert all(info[r]["status"] == 0 for r in range(5) if r != 2)
    X, info, st = plan.solve(dev(prob.V), opts=opts(ztoep.ZTOEP_FP64, 1e-12, max_iter=3), check=False)
    assert st == ztoep.ZTOEP_ERR_NOCONV
    assert all(i["inner_iters"] <= 3 for i in info)
    plan.close()


def test_solve_host_matches_device():
    prob = make("9x4_b40_e24")
    plan = ztoep.Plan.from_problem(prob)
    o = opts(ztoep.ZTOEP_MIXED, 1e-8)
    Xd, _, _ = plan.solve(dev(prob.V), opts=o)
    Vh = torch.from_numpy(prob.V.copy()).pin_memory()
    Xh = torch.zeros_like(Vh).pin_memory()
    o2 = opts(ztoep.ZTOEP_MIXED, 1e-8)
    o2.flags = ztoep.ZTOEP_FLAG_ZERO_GUESS
    info = ztoep.info_array(prob.nrhs)
    st = ztoep.ztoep_solve_host(plan.handle, o2, prob.nrhs, Vh, Xh, info)
    torch.cuda.synchronize()
    assert st == 0
    assert torch.equal(Xh, Xd.cpu())
    plan.close()


def test_initial_guess_is_used():
    prob = make("4x4_b8_e16")
    Z = oracle.assemble(prob)
    Xref = oracle.LU(Z).solve(prob.V)
    plan = ztoep.Plan.from_problem(prob)
    o = opts(ztoep.ZTOEP_FP64, 1e-10)
    X0 = dev(Xref)
    X, info, st = plan.solve(dev(prob.V), X=X0.clone(), opts=o)
    assert st == 0 and info[0]["inner_iters"] == 0 and info[0]["outer"] == 1
    plan.close()


def test_host_driven_loop_matches_graph_bitwise():
    prob = make("7x6_b12_e20")
    plan = ztoep.Plan.from_problem(prob)
    V = dev(prob.V)
    for prec in (ztoep.ZTOEP_MIXED, ztoep.ZTOEP_FP64):
        Xg, ig, _ = plan.solve(V, opts=opts(prec, 1e-9))
        o = opts(prec, 1e-9)
        o.flags = ztoep.ZTOEP_FLAG_HOST_LOOP
        Xh, ih, _ = plan.solve(V, opts=o)
        assert torch.equal(Xg, Xh)
        assert [i["inner_iters"] for i in ig] == [i["inner_iters"] for i in ih]


def test_timeout_is_enforced_on_device():
    prob = make("9x4_b40_e24")
    plan = ztoep.Plan.from_problem(prob)
    o = opts(ztoep.ZTOEP_FP64, 1e-14, max_iter=100000)
    o.max_outer = 100000
    o.timeout_ns = 1  # expires at the first check
    X, info, st = plan.solve(dev(prob.V), opts=o, check=False)
    assert st == ztoep.ZTOEP_ERR_TIMEOUT
    assert all(i["status"] == ztoep.ZTOEP_ERR_TIMEOUT for i in info)
    plan.close()


TC_CASES = [("9x4_b40_e24", 16), ("7x6_b12_e20", 20), ("6x6_b33_e0_gap", 33), ("3x5_b4_e12_pw3", 40),
            ("4x4_b8_e16", 17), ("9x4_b40_e24", 100), ("16x8_b32_e200", 24), ("16x8_b32_e200", 72)]
# shapes only the tensor-core tests use: several 128-row tiles of B and B^T,
# K split of B x_T into partial sums, RHS in chunks of 64
TC_EXTRA = {"16x8_b32_e200": dict(nx=16, ny=8, b=32, n_edge=200, seed=23)}


@pytest.mark.parametrize("key,nrhs", TC_CASES)
def test_matvec_mixed_tensor_core_path_vs_oracle(key, nrhs):
    # 16..256 RHS take the tcgen05 3xTF32 path for the block and edge products
    kw = dict(CASES[key] if key in CASES else TC_EXTRA[key])
    kw.update(rhs="planewave", nrhs=nrhs)
    prob = synth.make_problem(**kw)
    ref = oracle.matvec_dense(oracle.assemble(prob), prob.V)
    plan = ztoep.Plan.from_problem(prob)
    ztoep.ztoep_timing_reset()
    ztoep.ztoep_timing_enable(1 << ztoep.K_TENSOR | 1 << ztoep.K_TENSOR_PIPE)
    got = host(plan.matvec(dev(prob.V), ztoep.ZTOEP_MIXED))
    ztoep.ztoep_timing_enable(0)
    lockstep = ztoep.ztoep_timing_read(ztoep.K_TENSOR)[0]
    pipelined = ztoep.ztoep_timing_read(ztoep.K_TENSOR_PIPE)[0]
    assert lockstep + pipelined >= 1  # the tensor-core kernels ran
    if kw["b"] % 2 == 0 and (kw["nx"] * kw["ny"] * kw["b"] + kw["n_edge"]) % 2 == 0:
        assert lockstep == 0 and pipelined >= 2  # operands suit TMA: the pipelined kernel for every GEMM
    err = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-6
    plan.close()


def test_solve_mixed_tensor_core_path_vs_lu():
    kw = dict(CASES["9x4_b40_e24"])
    kw.update(rhs="planewave", nrhs=24)
    prob = synth.make_problem(**kw)
    Z = oracle.assemble(prob)
    Xref = oracle.LU(Z).solve(prob.V)
    plan = ztoep.Plan.from_problem(prob)
    X, info, st = plan.solve(dev(prob.V), opts=opts(ztoep.ZTOEP_MIXED, 1e-8))
    assert st == 0 and oracle.relres(Z, host(X), prob.V).max() <= 1e-8
    X2, _, st2 = plan.solve(dev(prob.V), opts=opts(ztoep.ZTOEP_MIXED, 1e-11))
    assert st2 == 0
    err = np.linalg.norm(host(X2) - Xref, axis=1) / np.linalg.norm(Xref, axis=1)
    assert err.max() <= 1e-7
    plan.close()
