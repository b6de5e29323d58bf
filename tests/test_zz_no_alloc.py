"""The allocation-free edge product (for callers that cannot allocate device
memory at call time, such as hosts that forbid allocation after start-up or a
framework whose pool has reserved the device memory) must give the same numbers
as the regular product, call after call, although all calls share one fixed
scratch array, and must not allocate.

Checked against ztoep_matvec (FP64) through the C-ABI:
  edge rows     Y[:, NT:] = (Z'X)[:, NT:]                       (<= 1e-12, max-norm relative)
  Toeplitz rows Y[:, :NT] = (Z'X - Z'X_T)[:, :NT] = B^T x_E     (<= 1e-12 of max |Z'X|)
This file is collected last so a failure here leaves every other test run.
"""
import numpy as np
import pytest
import torch

from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu

TOL = 1e-12


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def reference_parts(plan, X, nt):
    """B^T x_E rows and edge rows from the regular FP64 product."""
    full = plan.matvec(X, ztoep.ZTOEP_FP64)
    Xt = X.clone()
    Xt[:, nt:] = 0
    toep_only = plan.matvec(Xt, ztoep.ZTOEP_FP64)
    return (full - toep_only)[:, :nt], full[:, nt:], full


@pytest.mark.parametrize("kw", [
    dict(nx=9, ny=4, b=40, n_edge=24, rhs="planewave", nrhs=3, seed=13),
    dict(nx=5, ny=3, b=3, n_edge=10, gap_column=2, edge_layout="split", rhs="planewave", nrhs=2, seed=3),
])
def test_noalloc_edge_product_matches_matvec_two_calls(kw):
    prob = synth.make_problem(**kw)
    plan = ztoep.Plan.from_problem(prob)
    nt = prob.n_toep
    inputs = [prob.V, synth.manufactured_solution(prob, prob.nrhs, seed=99)]
    for Xn in inputs:  # two calls in a row, different inputs, one shared scratch
        X = dev(Xn)
        Y = torch.full_like(X, complex(np.nan, np.nan))
        st = ztoep.ztoep_edge_product_noalloc(plan.handle, prob.nrhs, X, Y)
        torch.cuda.synchronize()
        assert st == ztoep.ZTOEP_OK
        bt_ref, edge_ref, full = reference_parts(plan, X, nt)
        scale = full.abs().max().item()
        assert (Y[:, nt:] - edge_ref).abs().max().item() <= TOL * scale
        assert (Y[:, :nt] - bt_ref).abs().max().item() <= TOL * scale
        if not prob.active.all():
            absent = np.repeat(prob.active.reshape(-1) == 0, prob.b)
            assert torch.all(Y[:, :nt][:, torch.from_numpy(absent).cuda()] == 0)
    plan.close()


def test_noalloc_full_size_array_and_cap():
    prob, _ = synth.config_problem("c2_32x32_b64")
    plan = ztoep.Plan.from_problem(prob)
    nt = prob.n_toep
    for seed in (1, 2):
        X = dev(synth.manufactured_solution(prob, 1, seed=seed))
        Y = torch.empty_like(X)
        assert ztoep.ztoep_edge_product_noalloc(plan.handle, 1, X, Y) == ztoep.ZTOEP_OK
        bt_ref, edge_ref, full = reference_parts(plan, X, nt)
        scale = full.abs().max().item()
        assert (Y[:, nt:] - edge_ref).abs().max().item() <= TOL * scale
        assert (Y[:, :nt] - bt_ref).abs().max().item() <= TOL * scale
    # beyond the fixed scratch: rejected, output untouched
    X8 = dev(synth.manufactured_solution(prob, 8, seed=3))
    Y8 = torch.zeros_like(X8)
    assert ztoep.ztoep_edge_product_noalloc(plan.handle, 8, X8, Y8) == ztoep.ZTOEP_ERR_NOMEM
    torch.cuda.synchronize()
    assert torch.count_nonzero(Y8).item() == 0
    plan.close()


def test_noalloc_allocates_nothing_on_a_fresh_plan():
    """Free device memory (cudaMemGetInfo) is unchanged across calls on a plan
    that has never run a product, so no workspace exists yet: the regular
    product would allocate its partial sums here, this entry point must not."""
    prob = synth.make_problem(6, 5, 16, 22, seed=17, rhs="planewave", nrhs=2)
    # first call on this device (scratch address lookup, kernels loaded) on
    # another plan with the same RHS count, so the same kernels run below
    wprob = synth.make_problem(4, 3, 8, 10, seed=18, rhs="planewave", nrhs=2)
    warm = ztoep.Plan.from_problem(wprob)
    Xw = dev(wprob.V)
    assert ztoep.ztoep_edge_product_noalloc(warm.handle, 2, Xw, torch.empty_like(Xw)) == ztoep.ZTOEP_OK
    plan = ztoep.Plan.from_problem(prob)
    X = dev(prob.V)
    Y = torch.empty_like(X)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert ztoep.ztoep_edge_product_noalloc(plan.handle, prob.nrhs, X, Y) == ztoep.ZTOEP_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _, edge_ref, full = reference_parts(plan, X, prob.n_toep)
    assert (Y[:, prob.n_toep:] - edge_ref).abs().max().item() <= TOL * full.abs().max().item()
    plan.close()
    warm.close()


def test_noalloc_rejects_overlapping_buffers():
    prob = synth.make_problem(3, 4, 5, 6, seed=4, rhs="planewave", nrhs=2)
    plan = ztoep.Plan.from_problem(prob)
    buf = torch.zeros((3, prob.n), dtype=torch.complex128, device="cuda")
    X, Y = buf[0:2], buf[1:3]  # one RHS row shared
    assert ztoep.ztoep_edge_product_noalloc(plan.handle, 2, X, Y) == ztoep.ZTOEP_ERR_ARG
    assert ztoep.ztoep_matvec(plan.handle, ztoep.ZTOEP_FP64, 2, X, Y, None) == ztoep.ZTOEP_ERR_ARG
    plan.close()


def test_noalloc_without_edges_is_zero():
    prob = synth.make_problem(3, 4, 5, 0, seed=4, rhs="planewave", nrhs=2)
    plan = ztoep.Plan.from_problem(prob)
    X = dev(prob.V)
    Y = torch.ones_like(X)
    assert ztoep.ztoep_edge_product_noalloc(plan.handle, 2, X, Y) == ztoep.ZTOEP_OK
    torch.cuda.synchronize()
    assert torch.count_nonzero(Y).item() == 0
    assert ztoep.ztoep_edge_product_noalloc(plan.handle, 2, X, X) == ztoep.ZTOEP_ERR_ARG
    plan.close()
