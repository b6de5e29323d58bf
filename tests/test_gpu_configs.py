"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the benchmark uses (batched RHS, CUDA-graph solve).

The dense matrix is too large for an LU at these sizes (the 32x32 b64 system
would need 70 GB dense, the 64x64 b96 one 2.5 TB), so the oracle checks:
  - products on sampled rows, computed one by one from the generating blocks
    (FP64: <= 1e-12 of max |y|; MIXED: <= 2e-6 per RHS, 2-norm over the rows);
  - manufactured solutions: seeded X*, V = Z X* by the oracle, then the GPU
    solve must return X* to within cond(Z) x residual (bounds below);
  - true relative residuals recomputed by the oracle's direct product;
  - on the largest system, residual components on sampled rows
    (|r_k| <= tol ||v|| for every k follows from ||r|| <= tol ||v||).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def opts(prec, tol, restart=30):
    o = ztoep.ztoep_default_opts()
    o.prec, o.tol, o.restart = prec, tol, restart
    return o


def sample_rows(prob, count, seed=5):
    rng = np.random.default_rng(seed)
    rows = rng.choice(prob.n, size=min(count, prob.n), replace=False)
    edge = np.arange(prob.n_toep, prob.n)[:: max(1, prob.n_edge // 8)]
    return np.unique(np.concatenate([rows, edge, [0, prob.n_toep - 1, prob.n - 1]]))


def check_products_sampled(prob, plan, rows, X):
    ref = oracle.matvec_rows(prob, X, rows)
    Xd = dev(X)
    y64 = plan.matvec(Xd, ztoep.ZTOEP_FP64).cpu().numpy()[:, rows]
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * np.max(np.abs(ref))
    y32 = plan.matvec(Xd, ztoep.ZTOEP_MIXED).cpu().numpy()[:, rows]
    err = np.linalg.norm(y32 - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-6


def test_c1_fp64_gmres30_vs_lu():
    prob, tol = synth.config_problem("c1_4x4_b8")
    Z = oracle.assemble(prob)
    xref = oracle.LU(Z).solve(prob.V)
    plan = ztoep.Plan.from_problem(prob)
    X, info, st = plan.solve(dev(prob.V), opts=opts(ztoep.ZTOEP_FP64, tol))
    assert st == 0 and info[0]["rel_residual"] <= tol
    assert oracle.relres(Z, X.cpu().numpy(), prob.V).max() <= tol
    # cond_1(Z) ~ 5 here: forward error <= cond * residual
    err = np.linalg.norm(X.cpu().numpy() - xref) / np.linalg.norm(xref)
    assert err <= 1e-9
    plan.close()


@pytest.fixture(scope="module")
def c2():
    prob, tol = synth.config_problem("c2_32x32_b64")
    plan = ztoep.Plan.from_problem(prob)
    yield prob, tol, plan
    plan.close()


def test_c2_products_sampled_rows(c2):
    prob, tol, plan = c2
    rows = sample_rows(prob, 256)
    X = np.concatenate([prob.V, synth.manufactured_solution(prob, 1, seed=21)])
    check_products_sampled(prob, plan, rows, X)


@pytest.mark.parametrize("prec", [ztoep.ZTOEP_MIXED, ztoep.ZTOEP_FP64])
def test_c2_solve_config_rhs_and_manufactured(c2, prec):
    prob, tol, plan = c2
    # the configuration's RHS (broadside ones): true residual by the oracle
    X, info, st = plan.solve(dev(prob.V), opts=opts(prec, tol))
    assert st == 0
    res = oracle.relres(prob, X.cpu().numpy(), prob.V)
    assert res.max() <= tol and abs(res[0] - info[0]["rel_residual"]) <= 1e-3 * tol
    # manufactured solution: V = Z X* by the oracle, solved to 1e-10
    xs = synth.manufactured_solution(prob, 1, seed=77)
    V = oracle.matvec_blocks(prob, xs)
    X2, info2, st2 = plan.solve(dev(V), opts=opts(prec, 1e-10))
    assert st2 == 0
    err = np.linalg.norm(X2.cpu().numpy() - xs) / np.linalg.norm(xs)
    assert err <= 1e-7


def test_products_sampled_rows_wide_edge_ranges():
    """40x40 b64 array with 640 edge unknowns: more columns of [B | C] than
    one 128-column sub-tile per CTA of the FP32 edge kernel covers, so each CTA
    accumulates its row partials over two sub-tiles; 1 and 3 RHS."""
    prob = synth.make_problem(40, 40, 64, 640, seed=8, rhs="planewave", nrhs=3)
    plan = ztoep.Plan.from_problem(prob)
    rows = sample_rows(prob, 200)
    for r in (1, 3):
        check_products_sampled(prob, plan, rows, prob.V[:r])
    plan.close()


@pytest.fixture(scope="module")
def c3():
    prob, tol = synth.config_problem("c3_19x9gap_b48")
    plan = ztoep.Plan.from_problem(prob)
    Z = oracle.assemble(prob)
    yield prob, tol, plan, Z
    plan.close()


def test_c3_gap_products(c3):
    prob, tol, plan, Z = c3
    X = np.concatenate([prob.V[:4], synth.manufactured_solution(prob, 2, seed=31)])
    ref = oracle.matvec_dense(Z, X)
    y64 = plan.matvec(dev(X), ztoep.ZTOEP_FP64).cpu().numpy()
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_c3_162_ports_one_batched_solve(c3):
    prob, tol, plan, Z = c3
    assert prob.nrhs == 162 and prob.n == 8532
    X, info, st = plan.solve(dev(prob.V), opts=opts(ztoep.ZTOEP_MIXED, tol))
    assert st == 0
    Xh = X.cpu().numpy()
    res = oracle.relres(Z, Xh, prob.V)
    assert res.max() <= tol
    mask = oracle.unknown_mask(prob)
    assert np.all(Xh[:, mask == 0] == 0)  # the gap column stays exactly zero
    # manufactured solutions through the same batched path, solved to 1e-11
    xs = synth.manufactured_solution(prob, 16, seed=41)
    V = oracle.matvec_dense(Z, xs)
    X2, info2, st2 = plan.solve(dev(V), opts=opts(ztoep.ZTOEP_MIXED, 1e-11))
    assert st2 == 0
    err = np.linalg.norm(X2.cpu().numpy() - xs, axis=1) / np.linalg.norm(xs, axis=1)
    assert err.max() <= 1e-7


@pytest.mark.slow
def test_c4_64x64_b96_planewaves_sampled():
    prob, tol = synth.config_problem("c4_64x64_b96")
    assert prob.nrhs == 32 and prob.n == 394240
    plan = ztoep.Plan.from_problem(prob)
    rows = sample_rows(prob, 48)
    check_products_sampled(prob, plan, rows, prob.V[:4])
    X, info, st = plan.solve(dev(prob.V), opts=opts(ztoep.ZTOEP_MIXED, tol))
    assert st == 0
    assert max(i["rel_residual"] for i in info) <= tol
    Xh = X.cpu().numpy()
    r = prob.V[:, rows] - oracle.matvec_rows(prob, Xh, rows)
    vn = np.linalg.norm(prob.V, axis=1)
    assert np.all(np.abs(r) <= tol * vn[:, None])
    plan.close()


@pytest.mark.slow
def test_c4_64x64_b96_manufactured_both_precisions():
    """Full-size 64x64 b96 system (the tensor-core edge GEMMs, K split and the
    128-point passes at full size): V = Z x* by the oracle's direct product
    from the blocks, then both precisions solve it to 1e-10 and must return x*
    to 1e-7 (cond(Z) x residual)."""
    prob, _ = synth.config_problem("c4_64x64_b96")
    xs = synth.manufactured_solution(prob, 1, seed=64)
    V = oracle.matvec_blocks(prob, xs)
    plan = ztoep.Plan.from_problem(prob)
    for prec in (ztoep.ZTOEP_MIXED, ztoep.ZTOEP_FP64):
        X, info, st = plan.solve(dev(V), opts=opts(prec, 1e-10))
        assert st == 0 and info[0]["rel_residual"] <= 1e-10
        err = np.linalg.norm(X.cpu().numpy() - xs) / np.linalg.norm(xs)
        assert err <= 1e-7, (prec, err)
    plan.close()
