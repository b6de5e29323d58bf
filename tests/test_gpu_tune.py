"""Autotuner: a tuned plan computes the same product (to the parity bounds)
and solves to the tolerance; the choice is reused from the cache; a plan
built from an explicit choice gives bitwise the tuned plan's results; and a
RHS is summed identically alone and in a batch on a tuned plan."""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_04710_gb300 import synth, ztoep

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_products(prob, plan, X):
    ref = oracle.matvec_blocks(prob, X)
    Xd = dev(X)
    y64 = plan.matvec(Xd, ztoep.ZTOEP_FP64).cpu().numpy()
    assert np.max(np.abs(y64 - ref)) <= 1e-12 * np.max(np.abs(ref))
    y32 = plan.matvec(Xd, ztoep.ZTOEP_MIXED).cpu().numpy()
    err = np.linalg.norm(y32 - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert err.max() <= 2e-6


@pytest.mark.parametrize("nrhs", [3, 20])
def test_autotuned_plan_parity_and_cache(nrhs):
    prob = synth.make_problem(10, 6, 24, 40, seed=8, rhs="planewave", nrhs=nrhs)
    plan = ztoep.Plan.from_problem(prob, autotune=nrhs)
    t = plan.tune
    assert t.candidates > 1 and t.nrhs == nrhs
    assert 0 < t.product_us <= t.default_us
    assert t.lx >= 19 and t.ly >= 11 and plan.info.lx == t.lx and plan.info.ly == t.ly
    X = np.concatenate([prob.V, synth.manufactured_solution(prob, 2, seed=4)])
    check_products(prob, plan, X)
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-10
    Xs, info, st = plan.solve(dev(prob.V), opts=o)
    assert st == 0
    assert oracle.relres(prob, Xs.cpu().numpy(), prob.V).max() <= 1e-10
    # second call: from the cache, same choice
    plan2 = ztoep.Plan.from_problem(prob, autotune=nrhs)
    t2 = plan2.tune
    assert t2.candidates == 0
    for k in ("lx", "ly", "rad_order_x", "rad_order_y", "fft_channels_x", "fft_threads_x", "fft_channels_y",
              "fft_threads_y", "bp_split", "bp_ctas_per_sm", "tc_kchunk"):
        assert getattr(t2, k) == getattr(t, k), k
    # explicit choice: bitwise the same products and solution
    plan3 = ztoep.Plan.from_problem(prob, tune=t)
    Xd = dev(X)
    for prec in (ztoep.ZTOEP_FP64, ztoep.ZTOEP_MIXED):
        assert torch.equal(plan.matvec(Xd, prec), plan3.matvec(Xd, prec))
    Xs3, _, st3 = plan3.solve(dev(prob.V), opts=o)
    assert st3 == 0 and torch.equal(Xs, Xs3)
    got = ztoep.ztoep_plan_get_tune(plan3.handle)
    assert got.lx == t.lx and got.bp_split == t.bp_split
    for p in (plan, plan2, plan3):
        p.close()


def test_tuned_plan_batch_invariance():
    prob = synth.make_problem(7, 5, 16, 24, seed=21, rhs="planewave", nrhs=3)
    plan = ztoep.Plan.from_problem(prob, autotune=1)
    o = ztoep.ztoep_default_opts()
    o.tol = 1e-9
    Xb, _, st = plan.solve(dev(prob.V), opts=o)
    Xa, _, st1 = plan.solve(dev(prob.V[1:2]), opts=o)
    assert st == 0 and st1 == 0
    assert torch.equal(Xb[1:2], Xa)
    plan.close()


def test_bad_tune_rejected():
    prob = synth.make_problem(4, 4, 8, 8, seed=1)
    t = ztoep.TuneInfo()
    t.fft_threads_x = 100  # not a supported block size
    with pytest.raises(ztoep.ZtoepError):
        ztoep.Plan.from_problem(prob, tune=t)
    t = ztoep.TuneInfo()
    t.lx = 6  # below 2 nx - 1
    with pytest.raises(ztoep.ZtoepError):
        ztoep.Plan.from_problem(prob, tune=t)
