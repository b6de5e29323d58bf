"""Structured edge coupling (perimeter layout, side-Toeplitz B): the plan keeps
only the 2-D spectra of the 4k side generators and applies B and B^T in the
frequency domain.  The products must equal the oracle's dense products (FP64
<= 1e-12, mixed <= 2e-6 per RHS), solves must reach the oracle's LU solution,
the structured and dense plans must agree, and a B without the declared
structure (or an inconsistent descriptor) must be rejected."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SHAPES = [dict(nx=4, ny=4, b=8, k=1, seed=0), dict(nx=6, ny=5, b=12, k=2, seed=3),
          dict(nx=5, ny=7, b=6, k=3, seed=5), dict(nx=9, ny=4, b=40, k=1, seed=13),
          dict(nx=3, ny=2, b=33, k=4, seed=9), dict(nx=1, ny=1, b=4, k=2, seed=2),
          dict(nx=3, ny=3, b=70, k=8, seed=19), dict(nx=12, ny=10, b=20, k=4, seed=17)]


def make(sh, nrhs):
    return synth.make_problem(sh["nx"], sh["ny"], sh["b"], 2 * sh["k"] * (sh["nx"] + sh["ny"]), seed=sh["seed"],
                              rhs="planewave", nrhs=nrhs)


@pytest.mark.parametrize("sh", SHAPES, ids=lambda s: f"{s['nx']}x{s['ny']}_b{s['b']}_k{s['k']}")
@pytest.mark.parametrize("nrhs", [1, 3, 20])
def test_structured_products_match_dense_oracle(sh, nrhs):
    prob = make(sh, nrhs)
    X = np.concatenate([prob.V, synth.manufactured_solution(prob, 1, seed=7)])
    ref = oracle.matvec_dense(oracle.assemble(prob), X)
    plan = ztoep.Plan.from_problem(prob, structured=True)
    Xd = dev(X)
    y64 = plan.matvec(Xd, ztoep.ZTOEP_FP64).cpu().numpy()
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * np.max(np.abs(ref))
    y32 = plan.matvec(Xd, ztoep.ZTOEP_MIXED).cpu().numpy()
    err = np.linalg.norm(y32 - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-6
    plan.close()


@pytest.mark.parametrize("nrhs", [1, 13, 17])
def test_structured_products_many_tiles(nrhs):
    """32x32 cells (64x64 embedding: many CTA tiles and partial blocks of the
    fused side kernel, ragged RHS blocks) against the oracle's direct product."""
    prob = synth.make_problem(32, 32, 16, 2 * 4 * 64, seed=31, rhs="planewave", nrhs=nrhs)
    ref = oracle.matvec_blocks(prob, prob.V)
    plan = ztoep.Plan.from_problem(prob, structured=True)
    Xd = dev(prob.V)
    y64 = plan.matvec(Xd, ztoep.ZTOEP_FP64).cpu().numpy()
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * np.max(np.abs(ref))
    y32 = plan.matvec(Xd, ztoep.ZTOEP_MIXED).cpu().numpy()
    err = np.linalg.norm(y32 - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-6
    if nrhs < 16:  # same kernels alone and in the batch (16+ RHS: tensor-core block product)
        one = plan.matvec(Xd[nrhs - 1:], ztoep.ZTOEP_MIXED).cpu().numpy()
        assert np.array_equal(one[0], y32[nrhs - 1])
    plan.close()


@pytest.mark.parametrize("prec", [ztoep.ZTOEP_MIXED, ztoep.ZTOEP_FP64])
def test_structured_solve_vs_lu(prec):
    prob = make(SHAPES[1], 4)
    Z = oracle.assemble(prob)
    xref = oracle.LU(Z).solve(prob.V)
    plan = ztoep.Plan.from_problem(prob, structured=True)
    o = ztoep.ztoep_default_opts()
    o.prec, o.tol = prec, 1e-11
    X, info, st = plan.solve(dev(prob.V), opts=o)
    assert st == 0
    Xh = X.cpu().numpy()
    assert oracle.relres(Z, Xh, prob.V).max() <= 1e-11
    err = np.linalg.norm(Xh - xref, axis=1) / np.linalg.norm(xref, axis=1)
    assert err.max() <= 1e-8
    plan.close()


def test_structured_and_dense_plans_agree_and_structured_is_smaller():
    prob = make(SHAPES[3], 2)
    ps = ztoep.Plan.from_problem(prob, structured=True)
    pd = ztoep.Plan.from_problem(prob)
    X = dev(synth.manufactured_solution(prob, 2, seed=11))
    a, b = ps.matvec(X, ztoep.ZTOEP_FP64), pd.matvec(X, ztoep.ZTOEP_FP64)
    assert (a - b).abs().max().item() <= 1e-12 * b.abs().max().item()
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-10
    Xs, _, st1 = ps.solve(dev(prob.V), opts=o)
    Xd, _, st2 = pd.solve(dev(prob.V), opts=o)
    assert st1 == 0 and st2 == 0
    assert (Xs - Xd).abs().max().item() <= 1e-7 * Xd.abs().max().item()
    # no dense B resident
    assert ztoep.ztoep_plan_get_info(ps.handle).resident_bytes < ztoep.ztoep_plan_get_info(pd.handle).resident_bytes
    assert ztoep.ztoep_edge_product_noalloc(ps.handle, 1, X[:1], torch.empty_like(X[:1])) == \
        ztoep.ZTOEP_ERR_UNSUPPORTED
    ps.close()
    pd.close()


def test_structured_batch_invariance_and_host_loop():
    prob = make(SHAPES[2], 3)
    plan = ztoep.Plan.from_problem(prob, structured=True)
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-9
    Xb, _, st = plan.solve(dev(prob.V), opts=o)
    Xa, _, st1 = plan.solve(dev(prob.V[2:3]), opts=o)
    assert st == 0 and st1 == 0 and torch.equal(Xb[2:3], Xa)
    o2 = ztoep.ztoep_default_opts()
    o2.tol = 1e-9
    o2.flags = ztoep.ZTOEP_FLAG_HOST_LOOP
    Xh, _, st2 = plan.solve(dev(prob.V), opts=o2)
    assert st2 == 0 and torch.equal(Xb, Xh)
    plan.close()


def test_layout_that_does_not_hold_is_rejected():
    prob = make(SHAPES[1], 1)
    Bp = prob.B.copy()
    Bp[3, 17] *= 1.001  # one entry off the side-Toeplitz structure
    T, B, C = dev(prob.T), dev(Bp), dev(prob.C)
    with pytest.raises(ztoep.ZtoepError) as e:
        ztoep.Plan(prob.nx, prob.ny, prob.b, prob.n_edge, T, B, C, edge_per_cell=2)
    assert e.value.status == ztoep.ZTOEP_ERR_ARG
    with pytest.raises(ztoep.ZtoepError):  # n_edge inconsistent with the declared layout
        ztoep.Plan(prob.nx, prob.ny, prob.b, prob.n_edge, T, dev(prob.B), C, edge_per_cell=3)
    act = np.ones((prob.ny, prob.nx), np.uint8)
    act[1, 2] = 0
    with pytest.raises(ztoep.ZtoepError):  # absent elements are not supported with the layout
        ztoep.Plan(prob.nx, prob.ny, prob.b, prob.n_edge, T, dev(prob.B), C, active=act, edge_per_cell=2)
